// Fused tile kernel for the trigonometric bilateral filter (forward).
//
// One CTA owns a TH x TW tile of one channel of the output.  It reads the
// tile plus a halo of the spatial support from HBM once (clamp-to-edge), and
// then, for every term of the folded raised-cosine expansion (Section 2.3,
// eq. (final-form)):
//
//   phase 1: for each extended column j and each of cos / sin:
//              x(i) = cos|sin(omega f(i, j))                 (auxiliary image)
//              filter the pair (x, f*x) vertically -> V[cos|sin](:, j),
//                                                     V[f cos|f sin](:, j)
//            and keep a_m cos, a_m sin at the tile's own pixels;
//   phase 2: each thread owns a TWT-pixel row segment of either the
//            numerator P or the normaliser Q in registers, filters the pair
//            of planes it needs (cos part, sin part) horizontally and
//            accumulates
//              P += a_m cos(omega f(x)) W[f cos](x) + a_m sin(omega f(x)) W[f sin](x)
//              Q += a_m cos(omega f(x)) W[cos](x)   + a_m sin(omega f(x)) W[sin](x)
//
// and finally writes out = P / Q (Algorithm 1 step 5).  The auxiliary images
// never leave the SM; HBM sees one read of f and one write of out (and of Q
// when asked).  All arithmetic is FP32; the two planes of a pair share every
// filter instruction as one f32x2 operation (sm_100 and later).
//
// Spatial kernels (both separable, per axis):
//   KIND 0: truncated Gaussian, taps w[0 .. 2 RAD] from the kernel parameters;
//   KIND 1: three cascaded boxes of half-width RAD as running sums (Heckbert's
//           repeated integration done as cascaded box sums), unnormalised --
//           the common scale (2 RAD + 1)^-6 cancels in P / Q.
#pragma once

#include <cooperative_groups.h>
#include <cstdint>

#include "bf_internal.h"

namespace bf {

namespace cg = cooperative_groups;

// Most term groups of a tile (blocks of one cluster; above 8 a non-portable
// cluster size).
constexpr int kMaxTermSplit = 16;

constexpr float kTwoPi = 6.28318530717958647692f;

// sin(2 pi r) for r in turns: the argument is first reduced to [-1/2, 1/2]
// exactly (r - rint(r) is exact in FP32 for |r| < 2^23), so the hardware sine
// only ever sees [-pi, pi] however large omega f grows.
__device__ __forceinline__ float sin_turns(float r) {
    r = r - rintf(r);
    return __sinf(kTwoPi * r);
}

// ---- paired FP32 arithmetic (sm_100+: one instruction, two lanes of work) --
//
// The four auxiliary images of a term are filtered in pairs: (x, f x) in the
// vertical pass and (cos part, sin part) in the horizontal pass, so that every
// running-sum step, tap and accumulation of a pair is one f32x2 instruction.

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    unsigned long long d;
    const unsigned long long x = *reinterpret_cast<const unsigned long long *>(&a);
    const unsigned long long y = *reinterpret_cast<const unsigned long long *>(&b);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
    return *reinterpret_cast<const float2 *>(&d);
}

// Streamed 1-D filters on pairs.  Input k is produced by gen(k) right before
// the filter first needs it, and output k is handed to sink(k, y) as soon as
// it is complete, so only the filter's window is live in registers (all
// indices are compile-time after unrolling).

// Three cascaded boxes of half-width r (running sums, unnormalised):
// level l output k: s(k) = s(k - 1) + (in(k + 2r) - in(k - 1)).
template <int r, int NIN, class Gen, class Sink>
__device__ __forceinline__ void box3_stream(Gen &&gen, Sink &&sink) {
    constexpr int D = 2 * r;
    float2 a[NIN];
    float2 b[NIN - D];
    float2 c[NIN - 2 * D];
    float2 s1 = make_float2(0.f, 0.f), s2 = s1, s3 = s1;
#pragma unroll
    for (int i = 0; i < NIN; ++i) {
        a[i] = gen(i);
        if (i >= D) {
            const int k1 = i - D;
            if (k1 == 0) {
                s1 = a[0];
#pragma unroll
                for (int d = 1; d <= D; ++d) s1 = f2add(s1, a[d]);
            } else {
                s1 = f2add(s1, f2sub(a[k1 + D], a[k1 - 1]));
            }
            b[k1] = s1;
            if (k1 >= D) {
                const int k2 = k1 - D;
                if (k2 == 0) {
                    s2 = b[0];
#pragma unroll
                    for (int d = 1; d <= D; ++d) s2 = f2add(s2, b[d]);
                } else {
                    s2 = f2add(s2, f2sub(b[k2 + D], b[k2 - 1]));
                }
                c[k2] = s2;
                if (k2 >= D) {
                    const int k3 = k2 - D;
                    if (k3 == 0) {
                        s3 = c[0];
#pragma unroll
                        for (int d = 1; d <= D; ++d) s3 = f2add(s3, c[d]);
                    } else {
                        s3 = f2add(s3, f2sub(c[k3 + D], c[k3 - 1]));
                    }
                    sink(k3, s3);
                }
            }
        }
    }
}

// Truncated Gaussian taps w2[0 .. 2R] (each tap duplicated into both lanes).
template <int R, int NIN, class Gen, class Sink>
__device__ __forceinline__ void gauss_stream(Gen &&gen, Sink &&sink, const float2 *__restrict__ w2) {
    float2 a[NIN];
#pragma unroll
    for (int i = 0; i < NIN; ++i) {
        a[i] = gen(i);
        if (i >= 2 * R) {
            const int k = i - 2 * R;
            float2 acc = f2mul(w2[0], a[k]);
#pragma unroll
            for (int d = 1; d <= 2 * R; ++d) acc = f2fma(w2[d], a[k + d], acc);
            sink(k, acc);
        }
    }
}

template <int KIND, int RAD, int NIN, class Gen, class Sink>
__device__ __forceinline__ void filt2_stream(Gen &&gen, Sink &&sink, const float2 *__restrict__ w2) {
    if constexpr (KIND == 0) {
        gauss_stream<RAD, NIN>(gen, sink, w2);
    } else {
        box3_stream<RAD, NIN>(gen, sink);
    }
}

// NP pairs per step, streamed together (the backward pass filters (x, f x) and
// (f^2 x, 0) of one generated x in one sweep).
template <int NP>
struct Pairs {
    float2 v[NP];
};

template <int NP>
__device__ __forceinline__ Pairs<NP> padd(const Pairs<NP> &a, const Pairs<NP> &b) {
    Pairs<NP> c;
#pragma unroll
    for (int k = 0; k < NP; ++k) c.v[k] = f2add(a.v[k], b.v[k]);
    return c;
}

template <int NP>
__device__ __forceinline__ Pairs<NP> psub(const Pairs<NP> &a, const Pairs<NP> &b) {
    Pairs<NP> c;
#pragma unroll
    for (int k = 0; k < NP; ++k) c.v[k] = f2sub(a.v[k], b.v[k]);
    return c;
}

template <int r, int NIN, int NP, class Gen, class Sink>
__device__ __forceinline__ void box3_stream_n(Gen &&gen, Sink &&sink) {
    constexpr int D = 2 * r;
    Pairs<NP> a[NIN];
    Pairs<NP> b[NIN - D];
    Pairs<NP> c[NIN - 2 * D];
    Pairs<NP> s1, s2, s3;
#pragma unroll
    for (int i = 0; i < NIN; ++i) {
        a[i] = gen(i);
        if (i >= D) {
            const int k1 = i - D;
            if (k1 == 0) {
                s1 = a[0];
#pragma unroll
                for (int d = 1; d <= D; ++d) s1 = padd(s1, a[d]);
            } else {
                s1 = padd(s1, psub(a[k1 + D], a[k1 - 1]));
            }
            b[k1] = s1;
            if (k1 >= D) {
                const int k2 = k1 - D;
                if (k2 == 0) {
                    s2 = b[0];
#pragma unroll
                    for (int d = 1; d <= D; ++d) s2 = padd(s2, b[d]);
                } else {
                    s2 = padd(s2, psub(b[k2 + D], b[k2 - 1]));
                }
                c[k2] = s2;
                if (k2 >= D) {
                    const int k3 = k2 - D;
                    if (k3 == 0) {
                        s3 = c[0];
#pragma unroll
                        for (int d = 1; d <= D; ++d) s3 = padd(s3, c[d]);
                    } else {
                        s3 = padd(s3, psub(c[k3 + D], c[k3 - 1]));
                    }
                    sink(k3, s3);
                }
            }
        }
    }
}

template <int R, int NIN, int NP, class Gen, class Sink>
__device__ __forceinline__ void gauss_stream_n(Gen &&gen, Sink &&sink,
                                               const float2 *__restrict__ w2) {
    Pairs<NP> a[NIN];
#pragma unroll
    for (int i = 0; i < NIN; ++i) {
        a[i] = gen(i);
        if (i >= 2 * R) {
            const int k = i - 2 * R;
            Pairs<NP> acc;
#pragma unroll
            for (int q = 0; q < NP; ++q) acc.v[q] = f2mul(w2[0], a[k].v[q]);
#pragma unroll
            for (int d = 1; d <= 2 * R; ++d)
#pragma unroll
                for (int q = 0; q < NP; ++q) acc.v[q] = f2fma(w2[d], a[k + d].v[q], acc.v[q]);
            sink(k, acc);
        }
    }
}

template <int KIND, int RAD, int NIN, int NP, class Gen, class Sink>
__device__ __forceinline__ void filt2n_stream(Gen &&gen, Sink &&sink,
                                              const float2 *__restrict__ w2) {
    if constexpr (KIND == 0) {
        gauss_stream_n<RAD, NIN, NP>(gen, sink, w2);
    } else {
        box3_stream_n<RAD, NIN, NP>(gen, sink);
    }
}

// Generator adaptor for Pairs<NP> inputs, batches of GA as below.
template <int GA, int NIN, int NP, class Gen>
struct AheadN {
    Gen &g;
    Pairs<NP> buf[NIN];
    __device__ __forceinline__ explicit AheadN(Gen &gen) : g(gen) {}
    __device__ __forceinline__ Pairs<NP> operator()(int i) {
        if (i % GA == 0) {
#pragma unroll
            for (int d = 0; d < GA; ++d)
                if (i + d < NIN) buf[i + d] = g(i + d);
        }
        return buf[i];
    }
};

// Generator adaptor: produces the inputs in batches of GA so that their
// independent latency chains (shared-memory load, sine) overlap; measured
// faster than generating one input per step (too little to overlap) or all of
// them up front (too many registers).
constexpr int kGenAhead = 8;
template <int GA, int NIN, class Gen>
struct Ahead {
    Gen &g;
    float2 buf[NIN];
    __device__ __forceinline__ explicit Ahead(Gen &gen) : g(gen) {}
    __device__ __forceinline__ float2 operator()(int i) {
        if (i % GA == 0) {
#pragma unroll
            for (int d = 0; d < GA; ++d)
                if (i + d < NIN) buf[i + d] = g(i + d);
        }
        return buf[i];
    }
};

// ---- geometry --------------------------------------------------------------

template <int KIND, int RAD, int TH, int TW, int TWT>
struct TileGeom {
    static constexpr int HALO = KIND == 0 ? RAD : 3 * RAD;
    static constexpr int EH = TH + 2 * HALO;  // extended rows
    static constexpr int EW = TW + 2 * HALO;  // extended columns
    static constexpr int NSEG = TW / TWT;
    static constexpr int NT = TH * NSEG * 2;  // phase-2 threads: rows x segments x {P, Q}
    static constexpr int LN = TWT + 2 * HALO; // inputs of one phase-2 segment
    static constexpr int LN4 = (LN + 3) / 4;
    // f tile row stride (floats); rounded to a multiple of 4 for alignment
    static constexpr int SF = (EW + 3) / 4 * 4;
    // V row stride in floats (scalar kernels): covers every float4 a segment
    // reads, an odd number of float4s so that 8 consecutive rows hit 8
    // different 16-byte bank groups
    static constexpr int SV_MIN4 = (TW - TWT + 4 * LN4 + 3) / 4;
    static constexpr int SV = 4 * (SV_MIN4 % 2 ? SV_MIN4 : SV_MIN4 + 1);
    static constexpr int SC4 = TW / 4;
    static constexpr int SC = 4 * (SC4 % 2 ? SC4 : SC4 + 1);
    // Paired layout (forward): V2 rows of float2 {cos part, sin part}; the row
    // stride covers the columns phase 1 writes and the pairs of float2 that a
    // segment reads, and is 2 mod 4 float2 (an odd number of 16-byte units).
    static constexpr int LN2 = (LN + 1) / 2 * 2;
    static constexpr int SV2_MIN = (EW > TW - TWT + LN2 ? EW : TW - TWT + LN2);
    static constexpr int SV2 = (SV2_MIN + 3) / 4 * 4 + 2;
    static constexpr int SC2 = (TW + 3) / 4 * 4 + 2;
    static constexpr int F_FLOATS = EH * SF;
    static constexpr int V_FLOATS = 4 * TH * (SV > SV2 ? SV : SV2);
    static constexpr int C_FLOATS = 2 * TH * (SC > SC2 ? SC : SC2);
    static constexpr size_t SMEM = sizeof(float) * (size_t)(F_FLOATS + V_FLOATS + C_FLOATS);
    static_assert(TW % TWT == 0, "segments must tile the row");
    static_assert(TWT % 4 == 0 && TW % 4 == 0, "float4 access");
    static_assert(NT <= 1024, "block too large");
    static_assert(TH * SV <= V_FLOATS, "exchange buffer");
    static_assert(2 * EW <= NT, "one phase-1 item per thread");
};

struct TileParams {
    BfImage img;
    BfTerms terms;
    BfTaps taps;
    // Term split (small images): the terms are cut into `split` consecutive
    // groups, one block per tile and group, the groups of a tile launched as
    // one thread-block cluster; the cluster's first block sums the groups' P
    // and Q from the others' shared memory in group order and divides.
    // split = 1: all terms in one block, no cluster.
    int split;
};

// Everything one tile needs: the image, its term table and taps, the tile
// origin.  The term and tap arrays may live in kernel parameter space or in
// global memory.
struct TileJob {
    const void *in;   // this plane's first pixel
    float *out;       // this plane's first pixel
    float *q_out;
    long long in_row_stride;
    int H, W, in_px, out_px, dtype;
    float q_scale;
    const float *a;
    const float *t;
    int n_terms;
    const float2 *w2;  // Gaussian taps, each duplicated into a pair
    int x0, y0;
    // term groups of the tile (1: all terms in this block; > 1: this block
    // is one of a cluster of `split`, its rank the group)
    int split;
    // or, when not NULL: this block's terms are one group of a tile whose
    // groups run as separate work items; its P goes to slot (at the output's
    // offsets; Q slot_n further) for a later sum over the groups
    float *slot;
    long long slot_n;
};

// CLUSTER: the block is one term group of a cluster (TileJob::split > 1) and
// the epilogue reduces the cluster's groups; a separate instantiation, so
// that blocks holding all terms compile without that code.
template <int KIND, int RAD, int TH, int TW, int TWT, bool CLUSTER = false>
__device__ __forceinline__ void tile_body(const TileJob &jb, float *smem) {
    using G = TileGeom<KIND, RAD, TH, TW, TWT>;
    constexpr int HALO = G::HALO, EH = G::EH, EW = G::EW;
    constexpr int SV2 = G::SV2, SC2 = G::SC2;
    float *Fs = smem;
    // VP: vertically filtered {f cos, f sin}; VQ: {cos, sin} (float2 rows)
    float *VP = Fs + G::F_FLOATS;
    float *VQ = VP + 2 * TH * SV2;
    // CC: {a cos, a sin} at the tile's own pixels
    float *CC = Fs + G::F_FLOATS + G::V_FLOATS;

    const int tid = threadIdx.x;
    const int x0 = jb.x0, y0 = jb.y0;
    const int H = jb.H, W = jb.W;

    // ---- tile + halo of f, clamp-to-edge, converted to float
    for (int idx = tid; idx < EH * EW; idx += G::NT) {
        const int i = idx / EW;
        const int j = idx - i * EW;
        const int gy = min(max(y0 - HALO + i, 0), H - 1);
        const int gx = min(max(x0 - HALO + j, 0), W - 1);
        const long long off = (long long)gy * jb.in_row_stride + (long long)gx * jb.in_px;
        float v;
        if (jb.dtype == 0)
            v = __ldg(reinterpret_cast<const float *>(jb.in) + off);
        else
            v = (float)__ldg(reinterpret_cast<const uint8_t *>(jb.in) + off);
        Fs[i * G::SF + j] = v;
    }

    // phase-1 identity: item = (extended column j, q = cos | sin); adjacent
    // lanes take cos and sin of one column, so their stores are contiguous
    const int j1 = tid >> 1;
    const int q1 = tid & 1;
    const bool p1 = tid < 2 * EW;
    const bool own_col = j1 >= HALO && j1 < HALO + TW;
    const float ph0 = q1 ? 0.f : 0.25f;  // cos(t) = sin(t + quarter turn)
    // phase-2 identity: 8 consecutive lanes take 8 consecutive rows
    const int pi = tid % TH;
    const int rest = tid / TH;
    const int pa = rest & 1;   // 0: numerator P, 1: normaliser Q
    const int ps = rest >> 1;  // segment
    // P or Q of the segment's pixels (scalar: registers are the occupancy limit)
    float acc[TWT];
#pragma unroll
    for (int k = 0; k < TWT; ++k) acc[k] = 0.f;

    const int n_terms = jb.n_terms;
    for (int m = 0; m < n_terms; ++m) {
        __syncthreads();
        const float am = jb.a[m];
        const float tm = jb.t[m];
        // ---- phase 1: vertical filtering of (x, f x), x = cos | sin (omega f)
        if (p1) {
            const float *fcol = Fs + j1;
            float *ccol = CC + 2 * (j1 - HALO) + q1;
            float *vpcol = VP + 2 * j1 + q1;
            float *vqcol = VQ + 2 * j1 + q1;
            auto gen = [&](int i) {
                const float fv = fcol[i * G::SF];
                const float x = sin_turns(fmaf(tm, fv, ph0));
                if (i >= HALO && i < HALO + TH && own_col) ccol[(i - HALO) * 2 * SC2] = am * x;
                return make_float2(x, x * fv);
            };
            auto sink = [&](int k, float2 y) {
                vqcol[k * 2 * SV2] = y.x;
                vpcol[k * 2 * SV2] = y.y;
            };
            Ahead<kGenAhead, EH, decltype(gen)> ahead(gen);
            filt2_stream<KIND, RAD, EH>(ahead, sink, jb.w2);
        }
        __syncthreads();
        // ---- phase 2: horizontal filtering of (cos part, sin part) + combine
        {
            const float *vrow = (pa == 0 ? VP : VQ) + 2 * (pi * SV2 + ps * TWT);
            const float4 *src4 = reinterpret_cast<const float4 *>(vrow);
            const float4 *cc4 = reinterpret_cast<const float4 *>(CC + 2 * (pi * SC2 + ps * TWT));
            float4 ld[(G::LN + 1) / 2];
            float4 cl[TWT / 2];
            auto gen = [&](int i) {
                if ((i & 1) == 0) ld[i >> 1] = src4[i >> 1];
                const float4 v = ld[i >> 1];
                return (i & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
            };
            auto sink = [&](int k, float2 z) {
                if ((k & 1) == 0) cl[k >> 1] = cc4[k >> 1];
                const float4 c = cl[k >> 1];
                const float2 c2 = (k & 1) ? make_float2(c.z, c.w) : make_float2(c.x, c.y);
                acc[k] = fmaf(c2.x, z.x, fmaf(c2.y, z.y, acc[k]));
            };
            filt2_stream<KIND, RAD, G::LN>(gen, sink, jb.w2);
        }
    }

    // ---- out = P / Q
    __syncthreads();
    float *Xq = VP;  // Q of the tile's pixels (row stride G::SV)
    float *Xp = VQ;  // P, kept in shared memory only by term-split blocks
    if (jb.slot) {  // uniform: one term group's partial sums
        const int gy = y0 + pi;
        float *dstq = jb.slot + (pa == 1 ? jb.slot_n : 0);
#pragma unroll
        for (int k = 0; k < TWT; ++k) {
            const int gx = x0 + ps * TWT + k;
            if (gy < H && gx < W) dstq[((long long)gy * W + gx) * jb.out_px] = acc[k];
        }
        return;
    }
    if (pa == 1) {
#pragma unroll
        for (int k = 0; k < TWT; ++k) Xq[pi * G::SV + ps * TWT + k] = acc[k];
    } else if (CLUSTER) {
#pragma unroll
        for (int k = 0; k < TWT; ++k) Xp[pi * G::SV + ps * TWT + k] = acc[k];
    }
    __syncthreads();
    if constexpr (CLUSTER) {
        // the tile's term groups form one cluster: block g of the cluster
        // finishes the g-th slice of the tile's pixels, adding the groups' P
        // and Q (read from every block's shared memory) in group order
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        const int S = jb.split;
        const int g = (int)cl.block_rank();
        const int per = (TH * TW + S - 1) / S;
        for (int i = g * per + tid; i < min((g + 1) * per, TH * TW); i += G::NT) {
            const int row = i / TW, col = i - (i / TW) * TW;
            const int si = row * G::SV + col;
            float pr[kMaxTermSplit], qr[kMaxTermSplit];
#pragma unroll
            for (int r = 0; r < kMaxTermSplit; ++r)
                if (r < S) {
                    pr[r] = cl.map_shared_rank(Xp, r)[si];
                    qr[r] = cl.map_shared_rank(Xq, r)[si];
                }
            float pv = pr[0], qv = qr[0];
#pragma unroll
            for (int r = 1; r < kMaxTermSplit; ++r)
                if (r < S) {
                    pv += pr[r];
                    qv += qr[r];
                }
            const int gy = y0 + row, gx = x0 + col;
            if (gy < H && gx < W) {
                const long long o = ((long long)gy * W + gx) * jb.out_px;
                jb.out[o] = pv / qv;
                if (jb.q_out) jb.q_out[o] = qv * jb.q_scale;
            }
        }
        cl.sync();  // every block keeps its shared memory until the others have read it
        return;
    }
    if (pa == 0) {
        const int gy = y0 + pi;
        if (gy < H) {
#pragma unroll
            for (int k = 0; k < TWT; ++k) {
                const int gx = x0 + ps * TWT + k;
                if (gx < W) {
                    const float qv = Xq[pi * G::SV + ps * TWT + k];
                    const long long o = ((long long)gy * W + gx) * jb.out_px;
                    jb.out[o] = acc[k] / qv;
                    if (jb.q_out) jb.q_out[o] = qv * jb.q_scale;
                }
            }
        }
    }
}

// Resident blocks per SM the register allocation is sized for: one for the
// 512-thread blocks of the 64-row tiles, three for the 32 x 64 tiles of the
// smallest boxes (whose shared memory allows three and whose registers fit 80
// without spilling), two otherwise.
template <int KIND, int RAD, int TH, int TW>
struct TileMinBlocks {
    static constexpr int value = TH > 32 ? 1 : (KIND == 1 && RAD <= 2 && TW == 64) ? 3 : 2;
};

template <int KIND, int RAD, int TH, int TW, int TWT, bool CLUSTER>
__global__ void __launch_bounds__(TileGeom<KIND, RAD, TH, TW, TWT>::NT,
                                  TileMinBlocks<KIND, RAD, TH, TW>::value)
    bf_tile_fwd(const __grid_constant__ TileParams p) {
    extern __shared__ float4 smem4[];
    TileJob jb;
    // plane and term group (all terms, group 0, without a cluster)
    const int z = CLUSTER ? blockIdx.z / p.split : blockIdx.z;
    const int sg = CLUSTER ? blockIdx.z % p.split : 0;
    const int esz = p.img.dtype == 0 ? 4 : 1;
    jb.in = reinterpret_cast<const char *>(p.img.in) + (long long)z * p.img.in_z * esz;
    jb.out = p.img.out + (long long)z * p.img.out_z;
    jb.q_out = p.img.q_out ? p.img.q_out + (long long)z * p.img.out_z : nullptr;
    jb.in_row_stride = p.img.in_row_stride;
    jb.H = p.img.H;
    jb.W = p.img.W;
    jb.in_px = p.img.in_px;
    jb.out_px = p.img.out_px;
    jb.dtype = p.img.dtype;
    jb.q_scale = p.img.q_scale;
    const int nt = p.terms.n_terms;
    if constexpr (CLUSTER) {
        const int m0 = sg * nt / p.split, m1 = (sg + 1) * nt / p.split;
        jb.a = p.terms.a + m0;
        jb.t = p.terms.t + m0;
        jb.n_terms = m1 - m0;
    } else {
        jb.a = p.terms.a;
        jb.t = p.terms.t;
        jb.n_terms = nt;
    }
    jb.w2 = p.taps.w2;
    jb.x0 = blockIdx.x * TW;
    jb.y0 = blockIdx.y * TH;
    jb.split = CLUSTER ? p.split : 1;
    jb.slot = nullptr;
    jb.slot_n = 0;
    tile_body<KIND, RAD, TH, TW, TWT, CLUSTER>(jb, reinterpret_cast<float *>(smem4));
}

// The dynamic shared-memory opt-in of one kernel, once per device.
template <typename K>
cudaError_t tile_smem_attr(K kern, size_t smem, bool *done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !done[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) done[dev] = true;
    }
    return cudaSuccess;
}

// Launcher of the term-split (cluster) instantiation: prm.split > 1 groups of
// a tile's terms as one thread-block cluster.  Defined, and instantiated for
// every tile shape, in bf_tile_split.cu.
template <int KIND, int RAD, int TH, int TW, int TWT>
cudaError_t launch_tile_cluster(const TileParams &prm, cudaStream_t s);

template <int KIND, int RAD, int TH, int TW, int TWT>
cudaError_t launch_tile_cluster_impl(const TileParams &prm, cudaStream_t s) {
    using G = TileGeom<KIND, RAD, TH, TW, TWT>;
    auto kern = bf_tile_fwd<KIND, RAD, TH, TW, TWT, true>;
    static bool attr_set[64] = {}, big_cluster[64] = {};
    cudaError_t e = tile_smem_attr(kern, G::SMEM, attr_set);
    if (e != cudaSuccess) return e;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (prm.split > 8 && dev >= 0 && dev < 64 && !big_cluster[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        big_cluster[dev] = true;
    }
    // a tile's term groups (consecutive z) as one cluster
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((prm.img.W + TW - 1) / TW, (prm.img.H + TH - 1) / TH,
                       prm.img.C * prm.split);
    cfg.blockDim = dim3(G::NT);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = prm.split;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, prm);
}

// Host-side launcher for one instantiation (all terms per block, or the
// term-split cluster launch when prm.split > 1).
template <int KIND, int RAD, int TH, int TW, int TWT>
cudaError_t launch_tile(const TileParams &prm, cudaStream_t s) {
    using G = TileGeom<KIND, RAD, TH, TW, TWT>;
    if (prm.split > 1) return launch_tile_cluster<KIND, RAD, TH, TW, TWT>(prm, s);
    auto kern = bf_tile_fwd<KIND, RAD, TH, TW, TWT, false>;
    static bool attr_set[64] = {};
    cudaError_t e = tile_smem_attr(kern, G::SMEM, attr_set);
    if (e != cudaSuccess) return e;
    dim3 grid((prm.img.W + TW - 1) / TW, (prm.img.H + TH - 1) / TH, prm.img.C);
    kern<<<grid, G::NT, G::SMEM, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace bf

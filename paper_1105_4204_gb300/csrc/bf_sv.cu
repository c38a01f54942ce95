// Space-variant extension (Section 4): the range kernel stays fixed while the
// spatial kernel changes from pixel to pixel -- here pixel x averages over its
// own (2 r(x) + 1)^2 box, r(x) read from a radius map.  By eq. (final-form)
// this needs, per term, the space-variant box sums of the four auxiliary
// images, which summed-area tables give in O(1) per pixel (the box filter the
// section names; Crow's tables).
//
// One CTA owns a T x T output tile.  It reads the tile plus a halo of RM
// (clamp-to-edge) once and centres it: f~ = f - c, c the middle of the
// extended tile's range, h = max |f~| (the range kernel depends only on
// differences, so any per-tile offset gives the same filter; it halves the
// magnitude of the f-weighted planes).  Then, for every term m:
//   1. a thread per (plane, row) generates one row of one of the four planes
//        cos(w f~), sin(w f~), f~ cos(w f~), f~ sin(w f~)
//      over the extended tile (the sine as the cosine a quarter turn back),
//      converts each value to the fixed-point integer round(v 2^k) and keeps
//      its running sum along the row in a register, writing each table entry
//      once;
//   2. a thread per (plane, column) adds the rows up: four summed-area tables
//      in wrapping 32-bit arithmetic, row 0 and column 0 zero;
//   3. each own pixel reads its box sum of every plane from four entries of
//      its table and accumulates a_m (cos(w f~(x)) S[. cos] + sin(w f~(x))
//      S[. sin]) into Q (the plain planes) or P (the f~-weighted ones).
// out(x) = c + P / Q, with the fixed-point scales taken out as one power of
// two.
//
// Exactness.  Every plane value is |v| <= 1 (cos, sin) or |v| <= h (f~ cos,
// f~ sin).  The step 2^-k is chosen per plane pair so that |round(v 2^k)| <
// 2^21 and a box of (2 RM + 1)^2 values sums to less than 2^31 in magnitude:
// every box sum then comes out exact from the wrapping 32-bit tables, however
// large the prefix sums grow (no cancellation between large prefix sums, which
// in FP32 would lose the small boxes).  k is fixed by RM for the plain planes
// (2^-21 for boxes up to 17 x 17, 2^-20 up to 33 x 33) and set per tile from
// h for the weighted ones (2^-13 for a 33 x 33 box and h = 127.5); the
// rounding error per entry is then of the order of the FP32 sine's own.
// Rounding to the integer is one FMA against 1.5 * 2^23: the sum lands in
// [2^23, 2^24), where the FP32 spacing is 1, so the integer sits in the low
// mantissa bits.  The tables keep those bit patterns as they are; their
// constant part, 1.5 * 2^23's bit pattern per entry, is taken out of each box
// sum as (box area) x that pattern.
// Interleaved channels (H x W x C) are filtered independently with the same
// radius map, one grid z-slice per channel.
// HBM sees f and the radius map read once and out written once.
#include <cstdint>

#include "bf_internal.h"
#include "bf_tile.cuh"

namespace bf {

namespace {

constexpr float kSvMagic = 12582912.f;      // 1.5 * 2^23
constexpr unsigned kSvMagicBits = 0x4B400000u;  // its bit pattern
constexpr int kSvMaxQ = 21;                 // |round(v 2^k)| <= 2^21 < 2^22

struct SvParams {
    const void *in;
    long long in_stride;  // elements between rows
    int C;                // interleaved channels (blockIdx.z), in and out
    int dtype;            // 0 f32, 1 u8
    const int *radius;    // H x W, row-major
    int r_max;
    float *out;
    int H, W;
    BfTerms terms;
};

// Largest k <= 21 with 2^k * nbox below 2^31 (with a 0.1 % margin): the
// fixed-point exponent of the plain planes, |v| <= 1.
constexpr int sv_plain_exponent(int nbox) {
    int k = kSvMaxQ;
    while (k > 0 && (double)(1LL << k) * nbox >= 0.999 * 2147483648.0) --k;
    return k;
}

// Smallest n' >= n with n' = rem (mod 32): the table stride that puts the
// planes of a shared warp into disjoint banks (see the line layout below).
constexpr int sv_table_stride(int n, int rem) {
    if (rem == 0) return n;
    while (n % 32 != rem) ++n;
    return n;
}

template <int RM, int T, int NTHR, bool HAT>
struct SvGeom {
    static constexpr int E = T + 2 * RM;  // extended tile edge
    // Table entries per axis: the box's summed-area table has a zero row and
    // column first (E + 1); the hat's doubly integrated table two, and one
    // entry past the tile (E + 2).
    static constexpr int DT = E + (HAT ? 2 : 1);
    static constexpr int Z = HAT ? 2 : 1;  // leading zero rows and columns
    static constexpr int ES = DT | 1;      // table row stride: odd
    static constexpr int FS = E + 1;      // f~ tile row stride: odd, so that a thread
                                          // per row reads without bank conflicts
    // Table lines (a row in step 1, a column in step 2) go to threads in
    // blocks of 32 lines of one plane; the remaining E % 32 lines of the four
    // planes share warps, with the same line numbers in every plane (one
    // broadcast read of f~) and tables RMD banks apart.
    static constexpr int F = E / 32 * 32;  // lines per plane in whole warps
    static constexpr int RMD = E - F;      // remaining lines per plane
    static constexpr int TS = sv_table_stride(DT * ES, RMD);  // entries per table
    // the largest total weight of a pixel's kernel: (2 RM + 1)^2 boxes, or
    // (RM + 1)^4 for the hat of half-width RM
    static constexpr int NBOX = HAT ? (RM + 1) * (RM + 1) * (RM + 1) * (RM + 1)
                                    : (2 * RM + 1) * (2 * RM + 1);
    static constexpr int KQ = sv_plain_exponent(NBOX);
    static constexpr int OWN = T * T / NTHR;  // own pixels per thread
    static constexpr size_t SMEM = sizeof(unsigned) * 4 * TS + sizeof(float) * E * FS;
    static_assert(4 * E <= NTHR, "a thread per table row and per table column");
    static_assert(NTHR % T == 0 && NTHR % 32 == 0 && T % 32 == 0, "own-pixel layout");
    static_assert(RMD == 0 || 32 % RMD == 0, "whole planes of remaining lines per warp");
};

// 2^k for -126 <= k <= 127, exactly.
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

template <int RM, int T, int NTHR, bool HAT>
__global__ void __launch_bounds__(NTHR) bf_sv_fwd(const __grid_constant__ SvParams p) {
    using G = SvGeom<RM, T, NTHR, HAT>;
    constexpr int E = G::E, ES = G::ES, FS = G::FS, TS = G::TS, OWN = G::OWN, Z = G::Z;
    constexpr int NW = NTHR / 32;
    extern __shared__ unsigned sv_smem[];
    // tables 0 cos, 1 sin, 2 f~ cos, 3 f~ sin, then the E x E f~ tile
    unsigned *Tb = sv_smem;
    float *Fs = reinterpret_cast<float *>(Tb + 4 * TS);
    __shared__ float red[2][NW];

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * T, y0 = blockIdx.y * T;
    const int H = p.H, W = p.W;

    // ---- the extended tile, its range and its centre ----
    float mn = __int_as_float(0x7f800000), mx = -mn;
    for (int idx = tid; idx < E * E; idx += NTHR) {
        const int i = idx / E, j = idx - (idx / E) * E;
        const int gy = min(max(y0 - RM + i, 0), H - 1);
        const int gx = min(max(x0 - RM + j, 0), W - 1);
        const long long off = (long long)gy * p.in_stride + (long long)gx * p.C + blockIdx.z;
        const float v = p.dtype == 0 ? __ldg(reinterpret_cast<const float *>(p.in) + off)
                                     : (float)__ldg(reinterpret_cast<const uint8_t *>(p.in) + off);
        Fs[i * FS + j] = v;
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
    }
    for (int k = tid; k < G::DT; k += NTHR) {  // the leading zero rows and columns
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int z = 0; z < Z; ++z) {
                Tb[t * TS + z * ES + k] = 0u;
                Tb[t * TS + k * ES + z] = 0u;
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = mn;
        red[1][tid >> 5] = mx;
    }
    __syncthreads();
    mn = red[0][0];
    mx = red[1][0];
#pragma unroll
    for (int w = 1; w < NW; ++w) {
        mn = fminf(mn, red[0][w]);
        mx = fmaxf(mx, red[1][w]);
    }
    const float c = mn + 0.5f * (mx - mn);
    // fl(f - c) is monotone in f, so these two bound every centred value
    const float h = fmaxf(mx - c, c - mn);
    // weighted planes: largest 2^kp with h 2^kp <= min(2^21, 0.999 * 2^31 / NBOX)
    constexpr float kCap = (float)(0.999 * 2147483648.0 / G::NBOX) < (float)(1 << kSvMaxQ)
                               ? (float)(0.999 * 2147483648.0 / G::NBOX)
                               : (float)(1 << kSvMaxQ);
    const float lim = kCap / fmaxf(h, 1e-30f);
    const int kp = min(max((__float_as_int(lim) >> 23) - 127, -60), 60);  // floor(log2(lim))
    const float sP = pow2f(kp), sQ = pow2f(G::KQ);
    for (int idx = tid; idx < E * E; idx += NTHR) {
        const int i = idx / E, j = idx - (idx / E) * E;
        Fs[i * FS + j] -= c;
    }

    // own pixels: k-th of this thread at tile row tid / T + (NTHR / T) k, column tid % T
    int rad[OWN];
    float fo[OWN];
#pragma unroll
    for (int k = 0; k < OWN; ++k) {
        const int pi = tid / T + k * (NTHR / T), pj = tid % T;
        const int gy = y0 + pi, gx = x0 + pj;
        const int r = (gy < H && gx < W) ? __ldg(p.radius + (long long)gy * W + gx) : 0;
        rad[k] = min(max(r, 0), p.r_max);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < OWN; ++k) {
        const int pi = tid / T + k * (NTHR / T), pj = tid % T;
        fo[k] = Fs[(RM + pi) * FS + RM + pj];
    }

    float P[OWN], Q[OWN];
#pragma unroll
    for (int k = 0; k < OWN; ++k) P[k] = Q[k] = 0.f;

    // this thread's table line in steps 1 and 2: plane q, row (step 1) or column (step 2) l
    const bool line = tid < 4 * E;
    int q, l;
    if (tid < 4 * G::F) {
        q = tid / G::F;
        l = tid - q * G::F;
    } else {
        const int i = tid - 4 * G::F;
        q = G::RMD > 0 ? i / max(G::RMD, 1) : 0;
        l = G::F + i - q * G::RMD;
    }
    const float quarter = (q & 1) ? 0.25f : 0.f;  // sin(x) = cos(x - quarter turn)
    const bool weighted = q >= 2;

    for (int m = 0; m < p.terms.n_terms; ++m) {
        const float am = p.terms.a[m], tm = p.terms.t[m];
        // 1. one plane row: fixed point, running sum along the row
        if (line) {
            const float *frow = Fs + l * FS;
            auto value = [&](int j) {  // entry j of the row, biased fixed point
                const float fv = frow[j];
                float rr = __fmaf_rn(tm, fv, -quarter);
                rr = rr - rintf(rr);
                const float v = __cosf(kTwoPi * rr);
                const float s = weighted ? fv * sP : sQ;
                return __float_as_uint(__fmaf_rn(v, s, kSvMagic));
            };
            if constexpr (!HAT) {
                unsigned *row = Tb + q * TS + (l + 1) * ES + 1;
                unsigned run = 0u;
#pragma unroll 8
                for (int j = 0; j < E; ++j) {
                    run += value(j);
                    row[j] = run;
                }
            } else {
                // P2[t] = sum_{s < t} P1[s], P1[s] = sum_{j < s} v[j], t = 0 .. E + 1
                unsigned *row = Tb + q * TS + (l + 2) * ES;
                unsigned p1 = 0u, p2 = 0u;
#pragma unroll 8
                for (int j = 0; j < E; ++j) {
                    row[j] = p2;
                    p2 += p1;
                    p1 += value(j);
                }
                row[E] = p2;
                row[E + 1] = p2 + p1;
            }
        }
        __syncthreads();
        // 2. the columns: summed-area tables
        if (line) {
            if constexpr (!HAT) {
                unsigned *col = Tb + q * TS + ES + l + 1;
                unsigned run = 0u;
#pragma unroll 8
                for (int i = 0; i < E; ++i) {
                    run += col[i * ES];
                    col[i * ES] = run;
                }
            } else {
                // the same double integration down column l + 2, in place:
                // input row i sits at table row i + 2, output row t goes to row t
                unsigned *col = Tb + q * TS + l + 2;
                unsigned p1 = 0u, p2 = 0u;
#pragma unroll 8
                for (int i = 0; i < E; ++i) {
                    const unsigned in = col[(i + 2) * ES];
                    col[i * ES] = p2;
                    p2 += p1;
                    p1 += in;
                }
                col[E * ES] = p2;
                col[(E + 1) * ES] = p2 + p1;
            }
        }
        __syncthreads();
        // 3. box sums at the own pixels
#pragma unroll
        for (int k = 0; k < OWN; ++k) {
            const int pi = tid / T + k * (NTHR / T), pj = tid % T;
            // the own pixel's cos and sin, computed as its table entries are
            float rc = tm * fo[k];
            rc = rc - rintf(rc);
            float rs = __fmaf_rn(tm, fo[k], -0.25f);
            rs = rs - rintf(rs);
            const float cx = __cosf(kTwoPi * rc), sx = __cosf(kTwoPi * rs);
            const int r = rad[k];
            float S[4];
            if constexpr (!HAT) {
                const int a0 = (RM + pi - r) * ES, a1 = (RM + pi + r + 1) * ES;
                const int b0 = RM + pj - r, b1 = RM + pj + r + 1;
                const unsigned bias = (unsigned)((2 * r + 1) * (2 * r + 1)) * kSvMagicBits;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const unsigned *Tt = Tb + t * TS;
                    const unsigned s =
                        Tt[a1 + b1] - Tt[a0 + b1] - Tt[a1 + b0] + Tt[a0 + b0] - bias;
                    S[t] = __int2float_rn((int)s);
                }
            } else {
                // per axis, the hat of half-width r centred at c is the second
                // difference, step r + 1, of the doubly integrated table at c + 1
                const int ym = (RM + pi - r) * ES, yc = (RM + pi + 1) * ES;
                const int yp = (RM + pi + r + 2) * ES;
                const int xm = RM + pj - r, xc = RM + pj + 1, xp = RM + pj + r + 2;
                const unsigned m2 = (unsigned)((r + 1) * (r + 1));
                const unsigned bias = m2 * m2 * kSvMagicBits;  // the weights' sum, (r + 1)^4
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const unsigned *Tt = Tb + t * TS;
                    const unsigned corners = Tt[ym + xm] + Tt[ym + xp] + Tt[yp + xm] + Tt[yp + xp];
                    const unsigned edges = Tt[ym + xc] + Tt[yc + xm] + Tt[yc + xp] + Tt[yp + xc];
                    const unsigned s = corners - 2u * edges + 4u * Tt[yc + xc] - bias;
                    S[t] = __int2float_rn((int)s);
                }
            }
            Q[k] = __fmaf_rn(am, __fmaf_rn(cx, S[0], sx * S[1]), Q[k]);
            P[k] = __fmaf_rn(am, __fmaf_rn(cx, S[2], sx * S[3]), P[k]);
        }
        __syncthreads();  // the tables are rewritten next
    }
    // P is in units of 2^-kp, Q in units of 2^-KQ
    const float back = pow2f(G::KQ - kp);
#pragma unroll
    for (int k = 0; k < OWN; ++k) {
        const int pi = tid / T + k * (NTHR / T), pj = tid % T;
        const int gy = y0 + pi, gx = x0 + pj;
        if (gy < H && gx < W)
            p.out[((long long)gy * W + gx) * p.C + blockIdx.z] = c + P[k] / Q[k] * back;
    }
}

template <int RM, int T, int NTHR, bool HAT>
cudaError_t launch_sv(const SvParams &prm, cudaStream_t s) {
    using G = SvGeom<RM, T, NTHR, HAT>;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(bf_sv_fwd<RM, T, NTHR, HAT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    dim3 grid((prm.W + T - 1) / T, (prm.H + T - 1) / T, prm.C);
    bf_sv_fwd<RM, T, NTHR, HAT><<<grid, NTHR, G::SMEM, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace

int sv_max_radius(int hat) { return hat ? 8 : 16; }

cudaError_t launch_space_variant(const bf_plan *pl, const void *in, int dtype,
                                 long long row_stride, const int *radius, int r_max, int hat,
                                 float *out, int H, int W, int C, cudaStream_t s) {
    SvParams prm;
    prm.in = in;
    prm.in_stride = row_stride;
    prm.C = C;
    prm.dtype = dtype;
    prm.radius = radius;
    prm.r_max = r_max;
    prm.out = out;
    prm.H = H;
    prm.W = W;
    fill_terms(pl, &prm.terms);
    if (hat) {
        if (r_max <= 4) return launch_sv<4, 32, 256, true>(prm, s);
        if (r_max <= 8) return launch_sv<8, 32, 256, true>(prm, s);
        return cudaErrorInvalidValue;
    }
    if (r_max <= 4) return launch_sv<4, 32, 256, false>(prm, s);
    if (r_max <= 8) return launch_sv<8, 32, 256, false>(prm, s);
    return launch_sv<16, 64, 512, false>(prm, s);
}

}  // namespace bf

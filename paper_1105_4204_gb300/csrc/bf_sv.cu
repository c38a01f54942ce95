// Space-variant extension (Section 4): the range kernel stays fixed while the
// spatial kernel changes from pixel to pixel -- here pixel x averages over its
// own (2 r(x) + 1)^2 box, r(x) read from a radius map.  By eq. (final-form)
// this needs, per term, the space-variant box sums of the four auxiliary
// images, which summed-area tables give in O(1) per pixel (the box filter the
// section names; Crow's tables).
//
// One CTA owns a T x T output tile.  Its halo is the largest half-width R
// among its own pixels (so a tile of small boxes builds small tables; the
// launch's RM only bounds R and sizes the shared memory).  It reads the tile
// plus that halo (clamp-to-edge) once and centres it: f~ = f - c, c the
// middle of the extended tile's range, h = max |f~| (the range kernel depends
// only on differences, so any per-tile offset gives the same filter; it
// halves the magnitude of the f-weighted planes).  Then, for every term m:
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
// 2^21 and a box of (2 R + 1)^2 values sums to less than 2^31 in magnitude:
// every box sum then comes out exact from the wrapping 32-bit tables, however
// large the prefix sums grow (no cancellation between large prefix sums, which
// in FP32 would lose the small boxes).  k is set per tile: by R for the plain
// planes (2^-21 for boxes up to 17 x 17, 2^-20 up to 33 x 33) and by R and h
// for the weighted ones (2^-13 for a 33 x 33 box and h = 127.5); the rounding
// error per entry is then of the order of the FP32 sine's own.
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
__host__ __device__ constexpr int sv_plain_exponent(int nbox) {
    int k = kSvMaxQ;
    while (k > 0 && (double)(1LL << k) * nbox >= 0.999 * 2147483648.0) --k;
    return k;
}

// The largest total weight of a kernel of half-width r: (2 r + 1)^2 for the
// box, (r + 1)^4 for the hat.
__host__ __device__ constexpr int sv_nbox(int r, bool hat) {
    return hat ? (r + 1) * (r + 1) * (r + 1) * (r + 1) : (2 * r + 1) * (2 * r + 1);
}

// Smallest n' >= n with n' = rem (mod 32): the table stride that puts the
// planes of a shared warp into disjoint banks (see the line layout below).
constexpr int sv_table_stride(int n, int rem) {
    if (rem == 0) return n;
    while (n % 32 != rem) ++n;
    return n;
}

// Shared-memory layout for tiles with halos up to RM; a tile with halo R uses
// the leading T + 2 R (+ 1 or 2) rows and columns of each table.
template <int RM, int T, int NTHR, bool HAT>
struct SvGeom {
    static constexpr int E = T + 2 * RM;  // largest extended tile edge
    // Table entries per axis: the box's summed-area table has a zero row and
    // column first (E + 1); the hat's doubly integrated table two, and one
    // entry past the tile (E + 2).
    static constexpr int DT = E + (HAT ? 2 : 1);
    static constexpr int Z = HAT ? 2 : 1;  // leading zero rows and columns
    // The four tables share their rows: table row i holds row i of plane 0
    // at offset 0, of plane 2 at DT, of plane 1 at O1 and of plane 3 at
    // O1 + DT, O1 = 16 (mod 32), and rows are ES = 31 (mod 32) entries apart.
    // Then (a) a warp of 32 consecutive lines of one plane, or of the lines
    // a < 16 of planes q and q + 1 (the same for q + 2 and q + 3), spans the
    // 32 banks in steps 1 and 2; (b) in step 3 the entry at (row i + d, column
    // j + d) sits in the bank of (i, j): the corners (-r, -r) and
    // (r + 1, r + 1) of a lane's box fall in the bank of its own pixel whatever
    // its r, and the other two move by 2r + 1, so lanes of different radii
    // rarely meet in a bank.
    static constexpr int O1 = sv_table_stride(2 * DT, 16);
    static constexpr int ES = sv_table_stride(O1 + 2 * DT, 31);
    static constexpr int FS = E + 1;      // f~ tile row stride: odd, so that a thread
                                          // per row reads without bank conflicts
    static constexpr int OWN = T * T / NTHR;  // own pixels per thread
    static constexpr size_t SMEM = sizeof(unsigned) * DT * ES + sizeof(float) * E * FS;
    // offset of plane q within a table row
    static __device__ __forceinline__ constexpr int off(int q) {
        return (q & 1 ? O1 : 0) + (q >> 1) * DT;
    }
    static_assert(4 * E <= NTHR, "a thread per table row and per table column");
    // the box's carry lines (step 1 to step 2): entries per plane, 16 (mod 32)
    static constexpr int CY = sv_table_stride(E, 16);
    static_assert(NTHR % T == 0 && NTHR % 32 == 0 && T % 32 == 0, "own-pixel layout");
};

// 2^k for -126 <= k <= 127, exactly.
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

template <int RM, int T, int NTHR, bool HAT>
__global__ void __launch_bounds__(NTHR) bf_sv_fwd(const __grid_constant__ SvParams p) {
    using G = SvGeom<RM, T, NTHR, HAT>;
    constexpr int ES = G::ES, FS = G::FS, DT = G::DT, OWN = G::OWN, Z = G::Z;
    constexpr int NW = NTHR / 32;
    extern __shared__ unsigned sv_smem[];
    // tables 0 cos, 1 sin, 2 f~ cos, 3 f~ sin, then the f~ tile
    unsigned *Tb = sv_smem;
    float *Fs = reinterpret_cast<float *>(Tb + DT * ES);
    __shared__ float red[2][NW];
    __shared__ int redr[NW];
    // the box's first half-row totals per plane and row (plane q at
    // q CY), then a line of zeros
    constexpr int CY = G::CY;
    __shared__ unsigned Cy[HAT ? 1 : 5 * CY + 8];

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int x0 = blockIdx.x * T, y0 = blockIdx.y * T;
    const int H = p.H, W = p.W;

    // ---- own pixels' half-widths and the tile's halo R (their largest) ----
    // own pixel k of this thread: tile row tid / T + (NTHR / T) k, column tid % T
    int rad[OWN];
    int R = 0;
#pragma unroll
    for (int k = 0; k < OWN; ++k) {
        const int pi = tid / T + k * (NTHR / T), pj = tid % T;
        const int gy = y0 + pi, gx = x0 + pj;
        const int r = (gy < H && gx < W) ? __ldg(p.radius + (long long)gy * W + gx) : 0;
        rad[k] = min(max(r, 0), p.r_max);
        R = max(R, rad[k]);
    }
    R = __reduce_max_sync(0xffffffffu, R);
    if (lane == 0) redr[wid] = R;
    __syncthreads();
    R = redr[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) R = max(R, redr[w]);
    const int E = T + 2 * R;  // this tile's extended edge (<= G::E)
    if constexpr (!HAT)
        for (int k = tid; k < CY; k += NTHR) Cy[4 * CY + 8 + k] = 0u;
    for (int k = tid; k < G::DT; k += NTHR) {  // the leading zero rows and columns
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int z = 0; z < Z; ++z) {
                Tb[G::off(t) + z * ES + k] = 0u;
                Tb[G::off(t) + k * ES + z] = 0u;
            }
    }

    // ---- the extended tile, its range and its centre ----
    float mn = __int_as_float(0x7f800000), mx = -mn;
    for (int i = wid; i < E; i += NW) {
        const int gy = min(max(y0 - R + i, 0), H - 1);
        for (int j = lane; j < E; j += 32) {
            const int gx = min(max(x0 - R + j, 0), W - 1);
            const long long off = (long long)gy * p.in_stride + (long long)gx * p.C + blockIdx.z;
            const float v = p.dtype == 0
                                ? __ldg(reinterpret_cast<const float *>(p.in) + off)
                                : (float)__ldg(reinterpret_cast<const uint8_t *>(p.in) + off);
            Fs[i * FS + j] = v;
            mn = fminf(mn, v);
            mx = fmaxf(mx, v);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
        red[0][wid] = mn;
        red[1][wid] = mx;
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
    // plain planes: 2^kq by the tile's largest box; weighted planes: largest
    // 2^kp with h 2^kp <= min(2^21, 0.999 * 2^31 / nbox)
    const int nbox = sv_nbox(R, HAT);
    const int kq = sv_plain_exponent(nbox);
    const float cap = fminf(0.999f * 2147483648.f / (float)nbox, (float)(1 << kSvMaxQ));
    const float lim = cap / fmaxf(h, 1e-30f);
    const int kp = min(max((__float_as_int(lim) >> 23) - 127, -60), 60);  // floor(log2(lim))
    const float sP = pow2f(kp), sQ = pow2f(kq);
    for (int i = wid; i < E; i += NW)
        for (int j = lane; j < E; j += 32) Fs[i * FS + j] -= c;
    __syncthreads();

    float fo[OWN];
#pragma unroll
    for (int k = 0; k < OWN; ++k) {
        const int pi = tid / T + k * (NTHR / T), pj = tid % T;
        fo[k] = Fs[(R + pi) * FS + R + pj];
    }

    float P[OWN], Q[OWN];
#pragma unroll
    for (int k = 0; k < OWN; ++k) P[k] = Q[k] = 0.f;

    // this thread's column in step 2: plane q, column l.  Columns go to
    // threads in blocks of 32 of one plane; the remaining RMD = E % 32
    // columns of each plane go to warps of their own, planes q and q + 1 (q
    // even) in one warp when RMD <= 16, else a warp per plane (the table
    // layout keeps such warps free of bank conflicts).
    const int F = E / 32 * 32, RMD = E - F;
    const int PW = RMD <= 16 ? 2 : 1;  // planes per remainder warp
    bool line;
    int q, l;
    if (tid < 4 * F) {
        line = true;
        q = tid / F;
        l = tid - q * F;
    } else {
        const int i = tid - 4 * F, w = i >> 5, u = i & 31;
        const int v = u / max(RMD, 1);
        q = w * PW + v;
        l = F + u - v * RMD;
        line = RMD > 0 && v < PW && q < 4;
    }
    // step 1 takes a thread per (row l1, pair p1): the pair's plain plane p1
    // (cos or sin) and weighted plane p1 + 2 share one f~ read and one sine.
    // The box splits each row into two halves, (pair, half) k = 2 half + p1
    // taking the place of q above (the halves' offsets differ by a multiple
    // of 32 only when SL does; the layout argument holds per half); the hat
    // keeps whole rows: rows in blocks of 32 of one pair, the remaining rows
    // of both pairs in one warp when RMD <= 16, else a warp per pair.
    const int SL = (E + 1) / 2;  // the box's first half-row: columns [0, SL)
    bool line1;
    int p1, l1, half = 0;
    if constexpr (!HAT) {
        line1 = line;
        p1 = q & 1;
        half = q >> 1;
        l1 = l;
    } else if (tid < 2 * F) {
        line1 = true;
        p1 = tid / F;
        l1 = tid - p1 * F;
    } else {
        const int i = tid - 2 * F;
        p1 = i / max(RMD, 1);
        l1 = F + i - p1 * RMD;
        line1 = RMD > 0 && p1 < 2 && RMD <= 16;
        if (RMD > 16) {  // a warp per pair
            const int w = i >> 5, u = i & 31;
            p1 = w;
            l1 = F + u;
            line1 = w < 2 && u < RMD;
        }
    }
    const float quarter = p1 ? 0.25f : 0.f;  // sin(x) = cos(x - quarter turn)

    for (int m = 0; m < p.terms.n_terms; ++m) {
        const float am = p.terms.a[m], tm = p.terms.t[m];
        // 1. one row of a pair of planes: fixed point, running sums along the row
        if (line1) {
            const float *frow = Fs + l1 * FS;
            // entry j of the row in both planes, biased fixed point
            auto value = [&](int j, unsigned &u, unsigned &w) {
                const float fv = frow[j];
                float rr = __fmaf_rn(tm, fv, -quarter);
                rr = rr - rintf(rr);
                const float v = __cosf(kTwoPi * rr);
                u = __float_as_uint(__fmaf_rn(v, sQ, kSvMagic));
                w = __float_as_uint(__fmaf_rn(v, fv * sP, kSvMagic));
            };
            if constexpr (!HAT) {
                // running sums over this half of the row; the first half's
                // totals become the second half's carry, added in step 2
                const int j0 = half * SL, j1 = half ? E : SL;
                unsigned *row = Tb + G::off(p1) + (l1 + 1) * ES + 1;
                unsigned ru = 0u, rw = 0u;
#pragma unroll 8
                for (int j = j0; j < j1; ++j) {
                    unsigned u, w;
                    value(j, u, w);
                    ru += u;
                    rw += w;
                    row[j] = ru;
                    row[j + DT] = rw;
                }
                if (!half) {
                    Cy[p1 * CY + l1] = ru;
                    Cy[(p1 + 2) * CY + l1] = rw;
                }
            } else {
                // P2[t] = sum_{s < t} P1[s], P1[s] = sum_{j < s} v[j], t = 0 .. E + 1
                unsigned *row = Tb + G::off(p1) + (l1 + 2) * ES;
                unsigned u1 = 0u, u2 = 0u, w1 = 0u, w2 = 0u;
#pragma unroll 8
                for (int j = 0; j < E; ++j) {
                    row[j] = u2;
                    row[j + DT] = w2;
                    u2 += u1;
                    w2 += w1;
                    unsigned u, w;
                    value(j, u, w);
                    u1 += u;
                    w1 += w;
                }
                row[E] = u2;
                row[E + 1] = u2 + u1;
                row[E + DT] = w2;
                row[E + 1 + DT] = w2 + w1;
            }
        }
        __syncthreads();
        // 2. the columns: summed-area tables
        if (line) {
            if constexpr (!HAT) {
                // the second half's columns add the first half's row totals;
                // the first half's read a zero line (kept 8 banks from the
                // carries, so a warp spanning both halves reads without conflict)
                unsigned *col = Tb + G::off(q) + ES + l + 1;
                const unsigned *cy = Cy + (l < SL ? 4 * CY + 8 : q * CY);
                unsigned run = 0u;
#pragma unroll 8
                for (int i = 0; i < E; ++i) {
                    run += col[i * ES] + cy[i];
                    col[i * ES] = run;
                }
            } else {
                // the same double integration down column l + 2, in place:
                // input row i sits at table row i + 2, output row t goes to row t
                unsigned *col = Tb + G::off(q) + l + 2;
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
                const int a0 = (R + pi - r) * ES, a1 = (R + pi + r + 1) * ES;
                const int b0 = R + pj - r, b1 = R + pj + r + 1;
                const unsigned bias = (unsigned)((2 * r + 1) * (2 * r + 1)) * kSvMagicBits;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const unsigned *Tt = Tb + G::off(t);
                    const unsigned s =
                        Tt[a1 + b1] - Tt[a0 + b1] - Tt[a1 + b0] + Tt[a0 + b0] - bias;
                    S[t] = __int2float_rn((int)s);
                }
            } else {
                // per axis, the hat of half-width r centred at c is the second
                // difference, step r + 1, of the doubly integrated table at c + 1
                const int ym = (R + pi - r) * ES, yc = (R + pi + 1) * ES;
                const int yp = (R + pi + r + 2) * ES;
                const int xm = R + pj - r, xc = R + pj + 1, xp = R + pj + r + 2;
                const unsigned m2 = (unsigned)((r + 1) * (r + 1));
                const unsigned bias = m2 * m2 * kSvMagicBits;  // the weights' sum, (r + 1)^4
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const unsigned *Tt = Tb + G::off(t);
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
    // P is in units of 2^-kp, Q in units of 2^-kq
    const float back = pow2f(kq - kp);
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

// Space-variant extension (Section 4): the range kernel stays fixed while the
// spatial kernel changes from pixel to pixel -- here pixel x averages over its
// own (2 r(x) + 1)^2 box, r(x) read from a radius map.  By eq. (final-form)
// this needs, per term, the space-variant box sums of the four auxiliary
// images, which summed-area tables give in O(1) per pixel (the box filter the
// section names; Crow's tables).
//
// One CTA owns a kSvT x kSvT output tile.  It reads the tile plus a halo of RM
// (clamp-to-edge) once, then for every term:
//   1. generates the auxiliary planes (cos, sin, f cos, f sin) over the
//      extended tile and stores them as 64-bit fixed-point integers (value *
//      2^26, rounded) in tables whose row 0 and column 0 stay zero;
//   2. turns them into summed-area tables (running sums along rows, then
//      along columns, a thread per line);
//   3. reads each own pixel's box sums from four entries of each table and
//      accumulates a_m (cos(w f(x)) S[cos] + sin(w f(x)) S[sin]) into Q and
//      a_m (cos(w f(x)) S[f cos] + sin(w f(x)) S[f sin]) into P.
// The tables are built two at a time (NTAB = 2: (cos, sin), then (f cos,
// f sin), regenerating the sines): half the shared memory doubles the
// resident blocks, which measured faster than building all four at once
// (r_max = 8 on 2048^2: 3.31 vs 3.54 ms).
// Integer tables make every box sum exact for the fixed-point planes (no
// cancellation between large prefix sums, which in FP32 would lose the small
// boxes); the fixed-point step is 2^-26 (1.5e-8 of a unit plane value, below
// the FP32 sine's own error), and the largest table entry, 255 * 2^26 *
// (kSvT + 2 RM)^2 < 2^56, fits.  HBM sees f and the radius map read once and
// out written once.
#include <cstdint>

#include "bf_internal.h"
#include "bf_tile.cuh"

namespace bf {

namespace {

constexpr int kSvT = 32;         // output tile edge
constexpr int kSvThreads = 256;  // 4 own pixels per thread
constexpr float kSvScale = 67108864.f;            // 2^26
constexpr float kSvInvScale = 1.f / 67108864.f;   // 2^-26 (exact)

struct SvParams {
    const void *in;
    long long in_stride;  // elements between rows
    int dtype;            // 0 f32, 1 u8
    const int *radius;    // H x W, row-major
    int r_max;
    float *out;
    int H, W;
    BfTerms terms;
};

template <int RM, int NTAB>
struct SvGeom {
    static constexpr int E = kSvT + 2 * RM;  // extended tile edge
    static constexpr int ES = E + 1;         // table edge (zero row / column first)
    static constexpr size_t SMEM =
        sizeof(long long) * NTAB * ES * ES + sizeof(float) * E * E;
    static_assert(NTAB == 2 || NTAB == 4, "tables per pass");
    static_assert(NTAB * E <= kSvThreads, "a thread per table line");
};

template <int RM, int NTAB>
__global__ void __launch_bounds__(kSvThreads) bf_sv_fwd(const __grid_constant__ SvParams p) {
    using G = SvGeom<RM, NTAB>;
    constexpr int E = G::E, ES = G::ES;
    constexpr int TS = ES * ES;  // entries per table
    extern __shared__ long long sv_smem[];
    long long *Tb = sv_smem;                                     // NTAB tables
    float *Fs = reinterpret_cast<float *>(Tb + NTAB * TS);       // E x E extended f tile

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kSvT, y0 = blockIdx.y * kSvT;
    const int H = p.H, W = p.W;

    for (int idx = tid; idx < E * E; idx += kSvThreads) {
        const int i = idx / E, j = idx - (idx / E) * E;
        const int gy = min(max(y0 - RM + i, 0), H - 1);
        const int gx = min(max(x0 - RM + j, 0), W - 1);
        const long long off = (long long)gy * p.in_stride + gx;
        Fs[idx] = p.dtype == 0 ? __ldg(reinterpret_cast<const float *>(p.in) + off)
                               : (float)__ldg(reinterpret_cast<const uint8_t *>(p.in) + off);
    }
    for (int k = tid; k < ES; k += kSvThreads) {  // the zero row and column of every table
#pragma unroll
        for (int t = 0; t < NTAB; ++t) {
            Tb[t * TS + k] = 0;
            Tb[t * TS + k * ES] = 0;
        }
    }

    // own pixels: k-th of this thread at tile row (tid / 32) + 8 k, column tid % 32
    constexpr int kOwn = kSvT * kSvT / kSvThreads;
    int rad[kOwn];
    float fown[kOwn];
    bool ok[kOwn];
#pragma unroll
    for (int k = 0; k < kOwn; ++k) {
        const int pi = tid / kSvT + k * (kSvThreads / kSvT), pj = tid % kSvT;
        const int gy = y0 + pi, gx = x0 + pj;
        ok[k] = gy < H && gx < W;
        const int r = ok[k] ? __ldg(p.radius + (long long)gy * W + gx) : 0;
        rad[k] = min(max(r, 0), p.r_max);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kOwn; ++k) {
        const int pi = tid / kSvT + k * (kSvThreads / kSvT), pj = tid % kSvT;
        fown[k] = Fs[(RM + pi) * E + RM + pj];
    }

    float P[kOwn], Q[kOwn], cx[kOwn], sx[kOwn];
#pragma unroll
    for (int k = 0; k < kOwn; ++k) P[k] = Q[k] = 0.f;

    for (int m = 0; m < p.terms.n_terms; ++m) {
        const float am = p.terms.a[m], tm = p.terms.t[m];
#pragma unroll
        for (int k = 0; k < kOwn; ++k) {
            float rr = tm * fown[k];
            rr = rr - rintf(rr);
            __sincosf(kTwoPi * rr, &sx[k], &cx[k]);
        }
#pragma unroll 1
        for (int pass = 0; pass < 4 / NTAB; ++pass) {
            // 1. planes (pass * NTAB ...) of (cos, sin, f cos, f sin), fixed
            //    point, at table entry (i + 1, j + 1)
            for (int idx = tid; idx < E * E; idx += kSvThreads) {
                const int i = idx / E, j = idx - (idx / E) * E;
                const float fv = Fs[idx];
                float rr = tm * fv;
                rr = rr - rintf(rr);
                float sn, cs;
                __sincosf(kTwoPi * rr, &sn, &cs);
                long long *e0 = Tb + (i + 1) * ES + j + 1;
                if (NTAB == 4 || pass == 0) {
                    e0[0] = __float2ll_rn(cs * kSvScale);
                    e0[TS] = __float2ll_rn(sn * kSvScale);
                }
                if (NTAB == 4 || pass == 1) {
                    constexpr int o = NTAB == 4 ? 2 * TS : 0;
                    e0[o] = __float2ll_rn((cs * fv) * kSvScale);
                    e0[o + TS] = __float2ll_rn((sn * fv) * kSvScale);
                }
            }
            __syncthreads();
            // 2. summed-area tables: rows, then columns (a thread per line)
            if (tid < NTAB * E) {
                long long *row = Tb + (tid / E) * TS + (tid % E + 1) * ES;
                long long run = 0;
                for (int j = 1; j < ES; ++j) {
                    run += row[j];
                    row[j] = run;
                }
            }
            __syncthreads();
            if (tid < NTAB * E) {
                long long *col = Tb + (tid / E) * TS + tid % E + 1;
                long long run = 0;
                for (int i = 1; i < ES; ++i) {
                    run += col[i * ES];
                    col[i * ES] = run;
                }
            }
            __syncthreads();
            // 3. box sums at the own pixels
#pragma unroll
            for (int k = 0; k < kOwn; ++k) {
                const int pi = tid / kSvT + k * (kSvThreads / kSvT), pj = tid % kSvT;
                const int r = rad[k];
                const int a0 = RM + pi - r, a1 = RM + pi + r + 1;
                const int b0 = RM + pj - r, b1 = RM + pj + r + 1;
                float bs[NTAB];
#pragma unroll
                for (int t = 0; t < NTAB; ++t) {
                    const long long *T = Tb + t * TS;
                    const long long sum = T[a1 * ES + b1] - T[a0 * ES + b1] - T[a1 * ES + b0] +
                                          T[a0 * ES + b0];
                    bs[t] = __ll2float_rn(sum) * kSvInvScale;
                }
                const float vq = am * fmaf(cx[k], bs[0], sx[k] * bs[1]);
                if (NTAB == 4) {
                    Q[k] += vq;
                    P[k] += am * fmaf(cx[k], bs[2], sx[k] * bs[3]);
                } else if (pass == 0) {
                    Q[k] += vq;
                } else {
                    P[k] += vq;
                }
            }
            __syncthreads();  // the tables are rewritten next
        }
    }
#pragma unroll
    for (int k = 0; k < kOwn; ++k) {
        const int pi = tid / kSvT + k * (kSvThreads / kSvT), pj = tid % kSvT;
        if (ok[k]) p.out[(long long)(y0 + pi) * W + x0 + pj] = P[k] / Q[k];
    }
}

template <int RM, int NTAB>
cudaError_t launch_sv(const SvParams &prm, cudaStream_t s) {
    using G = SvGeom<RM, NTAB>;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(bf_sv_fwd<RM, NTAB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    dim3 grid((prm.W + kSvT - 1) / kSvT, (prm.H + kSvT - 1) / kSvT);
    bf_sv_fwd<RM, NTAB><<<grid, kSvThreads, G::SMEM, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace

int sv_max_radius() { return 16; }

cudaError_t launch_space_variant(const bf_plan *pl, const void *in, int dtype,
                                 long long row_stride, const int *radius, int r_max, float *out,
                                 int H, int W, cudaStream_t s) {
    SvParams prm;
    prm.in = in;
    prm.in_stride = row_stride;
    prm.dtype = dtype;
    prm.radius = radius;
    prm.r_max = r_max;
    prm.out = out;
    prm.H = H;
    prm.W = W;
    fill_terms(pl, &prm.terms);
    if (r_max <= 4) return launch_sv<4, 2>(prm, s);
    if (r_max <= 8) return launch_sv<8, 2>(prm, s);
    return launch_sv<16, 2>(prm, s);
}

}  // namespace bf

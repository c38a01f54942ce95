// Space-variant extension (Section 4): the range kernel stays fixed while the
// spatial kernel changes from pixel to pixel -- here pixel x averages over its
// own (2 r(x) + 1)^2 box, r(x) read from a radius map.  By eq. (final-form)
// this needs, per term, the space-variant box sums of the four auxiliary
// images, which summed-area tables give in O(1) per pixel (the box filter the
// section names; Crow's tables).
//
// One CTA owns a kSvT x kSvT output tile.  It reads the tile plus a halo of RM
// (clamp-to-edge) once, then for every term and for each of the two pairs
// (cos, sin) -> Q and (f cos, f sin) -> P:
//   1. generates the pair's planes over the extended tile and stores each
//      value as the fixed-point integer q = round(v * 2^26), split as
//      q = hi * 2^20 + lo (|hi| <= 2^14, |lo| <= 2^19), in two 32-bit tables
//      per plane whose row 0 and column 0 stay zero;
//   2. turns the four tables into summed-area tables (running sums along
//      rows, then along columns, a thread per line) in wrapping 32-bit
//      arithmetic;
//   3. reads each own pixel's box sums from four entries of each table --
//      exact, since a box of at most 33 x 33 keeps both halves' sums inside
//      32 bits -- and accumulates a_m (cos(w f(x)) S[. cos] + sin(w f(x))
//      S[. sin]) into Q or P.
// Integer tables make every box sum exact for the fixed-point planes (no
// cancellation between large prefix sums, which in FP32 would lose the small
// boxes); the fixed-point step is 2^-26 (1.5e-8 of a unit plane value, below
// the FP32 sine's own error).  The split into 32-bit halves is done with FP32
// additions (adding 1.5 * 2^23 to a float below 2^22 rounds it to the nearest
// integer and leaves that integer in its low mantissa bits), because
// conversions between FP32 and 64-bit integers run on the FP64 pipe, which
// on this GPU is narrow: with 64-bit tables they were the kernel's limit.
// HBM sees f and the radius map read once and out written once.
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

// round(v * 2^26) = hi * 2^20 + lo for |v| < 2^8, exactly, by FP32 additions.
__device__ __forceinline__ void fixed_split(float v, unsigned &hi, unsigned &lo) {
    constexpr float kM = 12582912.f;  // 1.5 * 2^23
    const float x = v * kSvScale;     // exact (a power of two)
    const float th = __fadd_rn(x * 9.5367431640625e-07f, kM);  // round(x / 2^20) + kM
    hi = (unsigned)(__float_as_int(th) - __float_as_int(kM));
    // x - round(x / 2^20) 2^20 is representable: the FMA is exact
    const float l = __fmaf_rn(-__fsub_rn(th, kM), 1048576.f, x);
    lo = (unsigned)(__float_as_int(__fadd_rn(l, kM)) - __float_as_int(kM));
}

template <int RM>
struct SvGeom {
    static constexpr int E = kSvT + 2 * RM;  // extended tile edge
    static constexpr int ES = E + 1;         // table edge (zero row / column first)
    static constexpr int NT = 4;             // tables per pass: (hi, lo) of two planes
    static constexpr size_t SMEM =
        sizeof(unsigned) * NT * ES * ES + sizeof(float) * E * E;
    static_assert(NT * E <= kSvThreads, "a thread per table line");
};

template <int RM>
__global__ void __launch_bounds__(kSvThreads) bf_sv_fwd(const __grid_constant__ SvParams p) {
    using G = SvGeom<RM>;
    constexpr int E = G::E, ES = G::ES, NT = G::NT;
    constexpr int TS = ES * ES;  // entries per table
    extern __shared__ unsigned sv_smem[];
    // tables: 0 hi / 1 lo of the pair's first plane, 2 hi / 3 lo of its second
    unsigned *Tb = sv_smem;
    float *Fs = reinterpret_cast<float *>(Tb + NT * TS);  // E x E extended f tile

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
        for (int t = 0; t < NT; ++t) {
            Tb[t * TS + k] = 0u;
            Tb[t * TS + k * ES] = 0u;
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
        for (int pass = 0; pass < 2; ++pass) {  // 0: (cos, sin) -> Q; 1: (f cos, f sin) -> P
            // 1. the pair's planes, fixed point, at table entry (i + 1, j + 1)
            for (int idx = tid; idx < E * E; idx += kSvThreads) {
                const int i = idx / E, j = idx - (idx / E) * E;
                const float fv = Fs[idx];
                float rr = tm * fv;
                rr = rr - rintf(rr);
                float sn, cs;
                __sincosf(kTwoPi * rr, &sn, &cs);
                if (pass == 1) {
                    cs = cs * fv;
                    sn = sn * fv;
                }
                unsigned *e0 = Tb + (i + 1) * ES + j + 1;
                fixed_split(cs, e0[0], e0[TS]);
                fixed_split(sn, e0[2 * TS], e0[3 * TS]);
            }
            __syncthreads();
            // 2. summed-area tables: rows, then columns (a thread per line)
            if (tid < NT * E) {
                unsigned *row = Tb + (tid / E) * TS + (tid % E + 1) * ES;
                unsigned run = 0u;
                for (int j = 1; j < ES; ++j) {
                    run += row[j];
                    row[j] = run;
                }
            }
            __syncthreads();
            if (tid < NT * E) {
                unsigned *col = Tb + (tid / E) * TS + tid % E + 1;
                unsigned run = 0u;
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
                float bs[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const unsigned *Th = Tb + (2 * q) * TS, *Tl = Th + TS;
                    const int sh = (int)(Th[a1 * ES + b1] - Th[a0 * ES + b1] - Th[a1 * ES + b0] +
                                         Th[a0 * ES + b0]);
                    const int sl = (int)(Tl[a1 * ES + b1] - Tl[a0 * ES + b1] - Tl[a1 * ES + b0] +
                                         Tl[a0 * ES + b0]);
                    bs[q] = fmaf(__int2float_rn(sh), 1048576.f, __int2float_rn(sl)) * kSvInvScale;
                }
                const float v = am * fmaf(cx[k], bs[0], sx[k] * bs[1]);
                if (pass == 0) Q[k] += v;
                else P[k] += v;
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

template <int RM>
cudaError_t launch_sv(const SvParams &prm, cudaStream_t s) {
    using G = SvGeom<RM>;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(bf_sv_fwd<RM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)G::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    dim3 grid((prm.W + kSvT - 1) / kSvT, (prm.H + kSvT - 1) / kSvT);
    bf_sv_fwd<RM><<<grid, kSvThreads, G::SMEM, s>>>(prm);
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
    if (r_max <= 4) return launch_sv<4>(prm, s);
    if (r_max <= 8) return launch_sv<8>(prm, s);
    return launch_sv<16>(prm, s);
}

}  // namespace bf

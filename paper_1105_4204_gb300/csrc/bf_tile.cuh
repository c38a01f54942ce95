// Fused tile kernel for the trigonometric bilateral filter (forward).
//
// One CTA owns a TH x TW tile of one channel of the output.  It reads the
// tile plus a halo of the spatial support from HBM once (clamp-to-edge), and
// then, for every term of the folded raised-cosine expansion (Section 2.3,
// eq. (final-form)):
//
//   phase 1: for each extended column j and each of cos / sin:
//              x(i) = cos|sin(omega f(i, j))                 (auxiliary image)
//              filter x vertically        -> V[cos|sin](:, j)
//              filter f*x vertically      -> V[f cos|f sin](:, j)
//            and keep a_m cos, a_m sin at the tile's own pixels;
//   phase 2: each thread owns a TWT-pixel row segment of either the
//            numerator P or the normaliser Q in registers, filters the two
//            planes it needs horizontally and accumulates
//              P += a_m cos(omega f(x)) W[f cos](x) + a_m sin(omega f(x)) W[f sin](x)
//              Q += a_m cos(omega f(x)) W[cos](x)   + a_m sin(omega f(x)) W[sin](x)
//
// and finally writes out = P / Q (Algorithm 1 step 5).  The auxiliary images
// never leave the SM; HBM sees one read of f and one write of out (and of Q
// when asked).  All arithmetic is FP32.
//
// Spatial kernels (both separable, per axis):
//   KIND 0: truncated Gaussian, taps w[0 .. 2 RAD] from the kernel parameters;
//   KIND 1: three cascaded boxes of half-width RAD as running sums (Heckbert's
//           repeated integration done as cascaded box sums), unnormalised --
//           the common scale (2 RAD + 1)^-6 cancels in P / Q.
#pragma once

#include <cstdint>

#include "bf_internal.h"

namespace bf {

constexpr float kTwoPi = 6.28318530717958647692f;

// sin(2 pi r) for r in turns: the argument is first reduced to [-1/2, 1/2]
// exactly (r - rint(r) is exact in FP32 for |r| < 2^23), so the hardware sine
// only ever sees [-pi, pi] however large omega f grows.
__device__ __forceinline__ float sin_turns(float r) {
    r = r - rintf(r);
    return __sinf(kTwoPi * r);
}

// ---- 1-D filters on register arrays (all indices compile-time) -------------

template <int R, int NIN>
__device__ __forceinline__ void gauss_taps(const float (&x)[NIN], float (&y)[NIN - 2 * R],
                                           const float *__restrict__ w) {
#pragma unroll
    for (int i = 0; i < NIN - 2 * R; ++i) {
        float acc = w[0] * x[i];
#pragma unroll
        for (int d = 1; d <= 2 * R; ++d) acc = fmaf(w[d], x[i + d], acc);
        y[i] = acc;
    }
}

template <int r, int NIN>
__device__ __forceinline__ void box_pass(const float (&x)[NIN], float (&y)[NIN - 2 * r]) {
    float s = x[0];
#pragma unroll
    for (int d = 1; d <= 2 * r; ++d) s += x[d];
    y[0] = s;
#pragma unroll
    for (int i = 1; i < NIN - 2 * r; ++i) {
        s += x[i + 2 * r] - x[i - 1];
        y[i] = s;
    }
}

template <int r, int NIN>
__device__ __forceinline__ void box3(const float (&x)[NIN], float (&y)[NIN - 6 * r]) {
    float t1[NIN - 2 * r];
    float t2[NIN - 4 * r];
    box_pass<r, NIN>(x, t1);
    box_pass<r, NIN - 2 * r>(t1, t2);
    box_pass<r, NIN - 4 * r>(t2, y);
}

template <int KIND, int RAD, int NIN>
struct Filt {
    static constexpr int HALO = KIND == 0 ? RAD : 3 * RAD;
    static constexpr int NOUT = NIN - 2 * HALO;
    __device__ __forceinline__ static void run(const float (&x)[NIN], float (&y)[NOUT],
                                               const float *__restrict__ w) {
        if constexpr (KIND == 0) {
            gauss_taps<RAD, NIN>(x, y, w);
        } else {
            box3<RAD, NIN>(x, y);
        }
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
    // V row stride: covers every float4 a segment reads, and is an odd number
    // of float4s so that 8 consecutive rows hit 8 different 16-byte bank groups
    static constexpr int SV_MIN4 = (TW - TWT + 4 * LN4 + 3) / 4;
    static constexpr int SV = 4 * (SV_MIN4 % 2 ? SV_MIN4 : SV_MIN4 + 1);
    static constexpr int SC4 = TW / 4;
    static constexpr int SC = 4 * (SC4 % 2 ? SC4 : SC4 + 1);
    static constexpr int F_FLOATS = EH * SF;
    static constexpr int V_FLOATS = 4 * TH * SV;
    static constexpr int C_FLOATS = 2 * TH * SC;
    static constexpr size_t SMEM = sizeof(float) * (size_t)(F_FLOATS + V_FLOATS + C_FLOATS);
    static_assert(TW % TWT == 0, "segments must tile the row");
    static_assert(TWT % 4 == 0 && TW % 4 == 0, "float4 access");
    static_assert(NT <= 1024, "block too large");
    static_assert(TH * SV <= V_FLOATS, "exchange buffer");
};

struct TileParams {
    BfImage img;
    BfTerms terms;
    BfTaps taps;
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
    const float *w;
    int x0, y0;
};

template <int KIND, int RAD, int TH, int TW, int TWT>
__device__ __forceinline__ void tile_body(const TileJob &jb, float *smem) {
    using G = TileGeom<KIND, RAD, TH, TW, TWT>;
    constexpr int HALO = G::HALO, EH = G::EH, EW = G::EW;
    float *Fs = smem;
    float *V = Fs + G::F_FLOATS;
    float *Cc = V + G::V_FLOATS;

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

    // phase-2 identity: 8 consecutive lanes take 8 consecutive rows
    const int pi = tid % TH;
    const int rest = tid / TH;
    const int pa = rest & 1;   // 0: numerator P, 1: normaliser Q
    const int ps = rest >> 1;  // segment
    float acc[TWT];
#pragma unroll
    for (int k = 0; k < TWT; ++k) acc[k] = 0.f;

    const int n_terms = jb.n_terms;
    for (int m = 0; m < n_terms; ++m) {
        __syncthreads();
        const float am = jb.a[m];
        const float tm = jb.t[m];
        // ---- phase 1: vertical filtering of the four auxiliary images
        for (int item = tid; item < 2 * EW; item += G::NT) {
            const int q = item >= EW ? 1 : 0;  // 0: cos, 1: sin
            const int j = item - q * EW;
            const float ph0 = q ? 0.f : 0.25f;  // cos(t) = sin(t + quarter turn)
            float x[EH];
#pragma unroll
            for (int i = 0; i < EH; ++i) x[i] = sin_turns(fmaf(tm, Fs[i * G::SF + j], ph0));
            if (j >= HALO && j < HALO + TW) {
                float *cdst = Cc + q * TH * G::SC + (j - HALO);
#pragma unroll
                for (int i = 0; i < TH; ++i) cdst[i * G::SC] = am * x[i + HALO];
            }
            float y[TH];
            Filt<KIND, RAD, EH>::run(x, y, jb.w);
            float *vdst = V + q * TH * G::SV + j;
#pragma unroll
            for (int i = 0; i < TH; ++i) vdst[i * G::SV] = y[i];
#pragma unroll
            for (int i = 0; i < EH; ++i) x[i] *= Fs[i * G::SF + j];
            Filt<KIND, RAD, EH>::run(x, y, jb.w);
            vdst += 2 * TH * G::SV;
#pragma unroll
            for (int i = 0; i < TH; ++i) vdst[i * G::SV] = y[i];
        }
        __syncthreads();
        // ---- phase 2: horizontal filtering + per-pixel combine
#pragma unroll
        for (int qq = 0; qq < 2; ++qq) {
            const int plane = (pa == 0 ? 2 : 0) + qq;
            const float4 *src =
                reinterpret_cast<const float4 *>(V + plane * TH * G::SV + pi * G::SV + ps * TWT);
            float yv[4 * G::LN4];
#pragma unroll
            for (int k = 0; k < G::LN4; ++k) {
                const float4 v4 = src[k];
                yv[4 * k] = v4.x;
                yv[4 * k + 1] = v4.y;
                yv[4 * k + 2] = v4.z;
                yv[4 * k + 3] = v4.w;
            }
            float yin[G::LN];
#pragma unroll
            for (int k = 0; k < G::LN; ++k) yin[k] = yv[k];
            float z[TWT];
            Filt<KIND, RAD, G::LN>::run(yin, z, jb.w);
            const float4 *cs =
                reinterpret_cast<const float4 *>(Cc + qq * TH * G::SC + pi * G::SC + ps * TWT);
#pragma unroll
            for (int k = 0; k < TWT / 4; ++k) {
                const float4 c4 = cs[k];
                acc[4 * k] = fmaf(c4.x, z[4 * k], acc[4 * k]);
                acc[4 * k + 1] = fmaf(c4.y, z[4 * k + 1], acc[4 * k + 1]);
                acc[4 * k + 2] = fmaf(c4.z, z[4 * k + 2], acc[4 * k + 2]);
                acc[4 * k + 3] = fmaf(c4.w, z[4 * k + 3], acc[4 * k + 3]);
            }
        }
    }

    // ---- out = P / Q
    __syncthreads();
    float *Xq = V;
    if (pa == 1) {
#pragma unroll
        for (int k = 0; k < TWT; ++k) Xq[pi * G::SV + ps * TWT + k] = acc[k];
    }
    __syncthreads();
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

template <int KIND, int RAD, int TH, int TW, int TWT>
__global__ void __launch_bounds__(TileGeom<KIND, RAD, TH, TW, TWT>::NT, 2)
    bf_tile_fwd(const __grid_constant__ TileParams p) {
    extern __shared__ float4 smem4[];
    TileJob jb;
    const int z = blockIdx.z;
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
    jb.a = p.terms.a;
    jb.t = p.terms.t;
    jb.n_terms = p.terms.n_terms;
    jb.w = p.taps.w;
    jb.x0 = blockIdx.x * TW;
    jb.y0 = blockIdx.y * TH;
    tile_body<KIND, RAD, TH, TW, TWT>(jb, reinterpret_cast<float *>(smem4));
}

// Host-side launcher for one instantiation.
template <int KIND, int RAD, int TH, int TW, int TWT>
cudaError_t launch_tile(const TileParams &prm, cudaStream_t s) {
    using G = TileGeom<KIND, RAD, TH, TW, TWT>;
    auto kern = bf_tile_fwd<KIND, RAD, TH, TW, TWT>;
    // the dynamic shared-memory opt-in is per device
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    dim3 grid((prm.img.W + TW - 1) / TW, (prm.img.H + TH - 1) / TH, prm.img.C);
    kern<<<grid, G::NT, G::SMEM, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace bf

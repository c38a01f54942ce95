// Fused adjoint (backward) tile kernel of the trigonometric bilateral filter.
//
// For L = sum_x u(x) out(x), out = P / Q of eq. (BF), alpha = u / Q and the
// folded raised cosine phi(s) = sum_m a_m cos(w_m s), the chain rule gives
// (with c_m(v) = cos(w_m v), s_m(v) = sin(w_m v), W the clamp-extended spatial
// filter and W^T its adjoint):
//
//   dL/df(p) = sum_m a_m w_m alpha_p [ c_p (W[f s] - o_p W[s]) - s_p (W[f c] - o_p W[c]) ](p)
//            + sum_m a_m [ c_p W^T[alpha c](p) + s_p W^T[alpha s](p) ]
//            - sum_m a_m w_m [ s_p (f_p W^T[alpha c] - W^T[alpha o c])
//                              - c_p (f_p W^T[alpha s] - W^T[alpha o s]) ](p)
//   dL/dsigma_r = (1/sigma_r) sum_p alpha_p sum_m a_m w_m
//                 { c_p [W[f^2 s] - (f_p + o_p) W[f s] + f_p o_p W[s]]
//                 - s_p [W[f^2 c] - (f_p + o_p) W[f c] + f_p o_p W[c]] }
//
// with N held fixed (phi depends on sigma_r through w_m = m / (sigma_r sqrt N)).
// The derivative of the range kernel is again a trigonometric sum (the paper's
// self-shiftability argument, Section 1), so the same on-chip plane machinery
// as the forward pass serves: per term, six clamp-extended planes
// (c, s, f c, f s, f^2 c, f^2 s) through W and four zero-extended planes
// (alpha c, alpha s, alpha o c, alpha o s) through W^T.  Per axis, W^T of the
// clamp-extended filter is the zero-extended filter with, at the first and
// last pixel, the tail mass folded back: W^T[g](0) = sum_{p=0..R} T(p) g(p),
// T(p) = sum_{d >= p} w1(d), and symmetrically at the last pixel.  The planes
// are recomputed from f, alpha and o; nothing but out and Q is kept from the
// forward pass.
#pragma once

#include "bf_tile.cuh"

namespace bf {

struct BwdParams {
    const float *f, *o, *q, *u;
    float *grad;         // dL/df, H x W per image; blockIdx.z selects the image of a stack
    double *partials;    // one dL/dsigma_r partial per block, or nullptr
    int H, W;
    long long img_stride;  // elements between consecutive images of a stack
    float scale;         // filter normalisation (box filters run unnormalised)
    float inv_sigma_r;
    BfTerms terms;       // a_m and turns per gray level
    float omega[BF_MAX_TERMS];  // w_m in radians per gray level
    BfTaps taps;
    float tail[2 * BF_MAX_TAPS_R + 1];  // T(p), p = 0 .. halo
    float total;         // sum of the 1-D taps (1 for the Gaussian, (2r+1)^3 for the box)
};

template <int KIND, int RAD, int TH, int TW, int TWT>
struct BwdGeom {
    static constexpr int HALO = KIND == 0 ? RAD : 3 * RAD;
    static constexpr int EH = TH + 2 * HALO;
    static constexpr int EW = TW + 2 * HALO;
    static constexpr int NSEG = TW / TWT;
    static constexpr int NT = TH * NSEG;
    static constexpr int LN = TWT + 2 * HALO;
    static constexpr int LN4 = (LN + 3) / 4;
    static constexpr int SF = (EW + 3) / 4 * 4;
    static constexpr int SV_MIN4 = (TW - TWT + 4 * LN4 + 3) / 4;
    static constexpr int SV = 4 * (SV_MIN4 % 2 ? SV_MIN4 : SV_MIN4 + 1);
    static constexpr int SC4 = TW / 4;
    static constexpr int SC = 4 * (SC4 % 2 ? SC4 : SC4 + 1);
    static constexpr int NPL = 6;  // planes held at once
    static constexpr int T_FLOATS = EH * SF;  // one extended tile
    static constexpr int V_FLOATS = NPL * TH * SV;
    static constexpr int C_FLOATS = 2 * TH * SC;
    static constexpr size_t SMEM =
        sizeof(float) * (size_t)(3 * T_FLOATS + V_FLOATS + C_FLOATS) + sizeof(double) * NT;
    static_assert(TW % TWT == 0 && TWT % 4 == 0, "segments");
    static_assert(NT <= 1024, "block");
};

template <int KIND, int RAD, int TH, int TW, int TWT>
__global__ void __launch_bounds__(BwdGeom<KIND, RAD, TH, TW, TWT>::NT)
    bf_tile_bwd(const __grid_constant__ BwdParams p) {
    using G = BwdGeom<KIND, RAD, TH, TW, TWT>;
    constexpr int HALO = G::HALO, EH = G::EH, EW = G::EW;
    extern __shared__ float4 smem4[];
    float *Fs = reinterpret_cast<float *>(smem4);  // f, clamp-extended
    float *As = Fs + G::T_FLOATS;                   // alpha, zero outside the image
    float *Os = As + G::T_FLOATS;                   // o, clamp-extended
    float *V = Os + G::T_FLOATS;                    // filtered planes
    float *Cc = V + G::V_FLOATS;                    // cos, sin at the tile's pixels
    double *red = reinterpret_cast<double *>(Cc + G::C_FLOATS);

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TW;
    const int y0 = blockIdx.y * TH;
    const int H = p.H, W = p.W;
    const long long zoff = (long long)blockIdx.z * p.img_stride;
    const float *pf = p.f + zoff, *po = p.o + zoff, *pq = p.q + zoff, *pu = p.u + zoff;
    float *pg = p.grad + zoff;

    for (int idx = tid; idx < EH * EW; idx += G::NT) {
        const int i = idx / EW;
        const int j = idx - i * EW;
        const int gyr = y0 - HALO + i, gxr = x0 - HALO + j;
        const int gy = min(max(gyr, 0), H - 1);
        const int gx = min(max(gxr, 0), W - 1);
        const size_t off = (size_t)gy * W + gx;
        const bool inside = gyr >= 0 && gyr < H && gxr >= 0 && gxr < W;
        Fs[i * G::SF + j] = __ldg(pf + off);
        Os[i * G::SF + j] = __ldg(po + off);
        As[i * G::SF + j] = inside ? __ldg(pu + off) / __ldg(pq + off) : 0.f;
    }

    const int pi = tid % TH;  // phase-2 row
    const int ps = tid / TH;  // phase-2 segment
    const int cx0 = ps * TWT;
    float gacc[TWT], sacc[TWT];
#pragma unroll
    for (int k = 0; k < TWT; ++k) gacc[k] = sacc[k] = 0.f;

    // border rows / columns of the image inside this tile (or -1)
    const int top = (y0 == 0) ? 0 : -1;                             // tile row of image row 0
    const int bot = (H - 1 >= y0 && H - 1 < y0 + TH) ? H - 1 - y0 : -1;
    const int lef = (x0 == 0) ? 0 : -1;
    const int rig = (W - 1 >= x0 && W - 1 < x0 + TW) ? W - 1 - x0 : -1;

    const int n_terms = p.terms.n_terms;
    for (int m = 0; m < n_terms; ++m) {
        const float am = p.terms.a[m];
        const float tm = p.terms.t[m];
        const float wm = p.omega[m];
        // ================= round A: W of c, s, f c, f s, f^2 c, f^2 s
        __syncthreads();
        for (int item = tid; item < 2 * EW; item += G::NT) {
            const int qq = item >= EW ? 1 : 0;
            const int j = item - qq * EW;
            const float ph0 = qq ? 0.f : 0.25f;
            float x[EH];
#pragma unroll
            for (int i = 0; i < EH; ++i) x[i] = sin_turns(fmaf(tm, Fs[i * G::SF + j], ph0));
            if (j >= HALO && j < HALO + TW) {
                float *cd = Cc + qq * TH * G::SC + (j - HALO);
#pragma unroll
                for (int i = 0; i < TH; ++i) cd[i * G::SC] = x[i + HALO];
            }
            float y[TH];
#pragma unroll 1
            for (int pw = 0; pw < 3; ++pw) {
                if (pw > 0) {
#pragma unroll
                    for (int i = 0; i < EH; ++i) x[i] *= Fs[i * G::SF + j];
                }
                Filt<KIND, RAD, EH>::run(x, y, p.taps.w);
                float *vd = V + (2 * pw + qq) * TH * G::SV + j;
#pragma unroll
                for (int i = 0; i < TH; ++i) vd[i * G::SV] = y[i];
            }
        }
        __syncthreads();
        {
            // per-pixel factors k c = a w alpha c, k s = a w alpha s, f, o
            float kc[TWT], ks[TWT], fp[TWT], op[TWT];
#pragma unroll
            for (int k = 0; k < TWT; ++k) {
                const int ti = (pi + HALO) * G::SF + cx0 + k + HALO;
                const float kk = am * wm * As[ti];
                kc[k] = kk * Cc[pi * G::SC + cx0 + k];
                ks[k] = kk * Cc[TH * G::SC + pi * G::SC + cx0 + k];
                fp[k] = Fs[ti];
                op[k] = Os[ti];
            }
#pragma unroll 1
            for (int pl = 0; pl < 6; ++pl) {
                const float4 *src = reinterpret_cast<const float4 *>(V + pl * TH * G::SV +
                                                                     pi * G::SV + cx0);
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
                Filt<KIND, RAD, G::LN>::run(yin, z, p.taps.w);
                // this plane's weights in dL/df (gc) and dL/dsigma_r (sc)
                float gc[TWT], sc[TWT];
                switch (pl) {
                    case 0:  // W[c]
#pragma unroll
                        for (int k = 0; k < TWT; ++k) {
                            gc[k] = ks[k] * op[k];
                            sc[k] = -ks[k] * fp[k] * op[k];
                        }
                        break;
                    case 1:  // W[s]
#pragma unroll
                        for (int k = 0; k < TWT; ++k) {
                            gc[k] = -kc[k] * op[k];
                            sc[k] = kc[k] * fp[k] * op[k];
                        }
                        break;
                    case 2:  // W[f c]
#pragma unroll
                        for (int k = 0; k < TWT; ++k) {
                            gc[k] = -ks[k];
                            sc[k] = ks[k] * (fp[k] + op[k]);
                        }
                        break;
                    case 3:  // W[f s]
#pragma unroll
                        for (int k = 0; k < TWT; ++k) {
                            gc[k] = kc[k];
                            sc[k] = -kc[k] * (fp[k] + op[k]);
                        }
                        break;
                    case 4:  // W[f^2 c]
#pragma unroll
                        for (int k = 0; k < TWT; ++k) {
                            gc[k] = 0.f;
                            sc[k] = -ks[k];
                        }
                        break;
                    default:  // W[f^2 s]
#pragma unroll
                        for (int k = 0; k < TWT; ++k) {
                            gc[k] = 0.f;
                            sc[k] = kc[k];
                        }
                        break;
                }
#pragma unroll
                for (int k = 0; k < TWT; ++k) {
                    gacc[k] = fmaf(gc[k], z[k], gacc[k]);
                    sacc[k] = fmaf(sc[k], z[k], sacc[k]);
                }
            }
        }
        // ================= round B: W^T of alpha c, alpha s, alpha o c, alpha o s
        __syncthreads();
        for (int item = tid; item < 2 * EW; item += G::NT) {
            const int qq = item >= EW ? 1 : 0;
            const int j = item - qq * EW;
            const float ph0 = qq ? 0.f : 0.25f;
            float x[EH];
#pragma unroll
            for (int i = 0; i < EH; ++i)
                x[i] = As[i * G::SF + j] * sin_turns(fmaf(tm, Fs[i * G::SF + j], ph0));
            float y[TH];
#pragma unroll 1
            for (int pw = 0; pw < 2; ++pw) {
                if (pw > 0) {
#pragma unroll
                    for (int i = 0; i < EH; ++i) x[i] *= Os[i * G::SF + j];
                }
                Filt<KIND, RAD, EH>::run(x, y, p.taps.w);
                float *vd = V + (2 * pw + qq) * TH * G::SV + j;
#pragma unroll
                for (int i = 0; i < TH; ++i) vd[i * G::SV] = y[i];
                // tail fold at the image's first / last row (a one-row image
                // keeps the whole mass on its only row)
                if (top >= 0 && bot == top) {
                    vd[top * G::SV] = p.total * x[HALO];
                } else if (top >= 0) {
                    float acc = 0.f;
#pragma unroll
                    for (int d = 0; d <= HALO; ++d) acc = fmaf(p.tail[d], x[HALO + d], acc);
                    vd[top * G::SV] = acc;
                }
                if (bot >= 0 && bot != top) {
                    // image row H-1-d sits at extended row bot + HALO - d (>= 0)
                    float acc = 0.f;
                    for (int d = 0; d <= HALO; ++d) {
                        const int i = bot + HALO - d;
                        float g = As[i * G::SF + j] * sin_turns(fmaf(tm, Fs[i * G::SF + j], ph0));
                        if (pw > 0) g *= Os[i * G::SF + j];
                        acc = fmaf(p.tail[d], g, acc);
                    }
                    vd[bot * G::SV] = acc;
                }
            }
        }
        __syncthreads();
        {
            float ca[TWT], cb[TWT], cc[TWT], cd[TWT];
#pragma unroll
            for (int k = 0; k < TWT; ++k) {
                const int ti = (pi + HALO) * G::SF + cx0 + k + HALO;
                const float c = Cc[pi * G::SC + cx0 + k];
                const float s = Cc[TH * G::SC + pi * G::SC + cx0 + k];
                const float fv = Fs[ti];
                const float aw = am * wm;
                ca[k] = am * c - aw * s * fv;  // W^T[alpha c]
                cb[k] = am * s + aw * c * fv;  // W^T[alpha s]
                cc[k] = aw * s;                // W^T[alpha o c]
                cd[k] = -aw * c;               // W^T[alpha o s]
            }
#pragma unroll 1
            for (int pl = 0; pl < 4; ++pl) {
                const float *row = V + pl * TH * G::SV + pi * G::SV;
                const float4 *src = reinterpret_cast<const float4 *>(row + cx0);
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
                Filt<KIND, RAD, G::LN>::run(yin, z, p.taps.w);
                // tail fold at the image's first / last column
                if (lef >= 0 && rig == 0 && cx0 == 0) {
                    z[0] = p.total * row[HALO];
                } else if (lef >= 0 && cx0 == 0) {
                    float acc = 0.f;
#pragma unroll
                    for (int d = 0; d <= HALO; ++d) acc = fmaf(p.tail[d], row[HALO + d], acc);
                    z[0] = acc;
                }
                if (rig >= cx0 && rig < cx0 + TWT && !(lef >= 0 && rig == 0)) {
                    float acc = 0.f;
                    for (int d = 0; d <= HALO; ++d) acc = fmaf(p.tail[d], row[rig + HALO - d], acc);
#pragma unroll
                    for (int k = 0; k < TWT; ++k)
                        if (k == rig - cx0) z[k] = acc;
                }
#pragma unroll
                for (int k = 0; k < TWT; ++k) {
                    const float cf = pl == 0 ? ca[k] : pl == 1 ? cb[k] : pl == 2 ? cc[k] : cd[k];
                    gacc[k] = fmaf(cf, z[k], gacc[k]);
                }
            }
        }
    }

    // ---- outputs: dL/df, and this block's share of dL/dsigma_r
    const int gy = y0 + pi;
    double sl = 0.0;
#pragma unroll
    for (int k = 0; k < TWT; ++k) {
        const int gx = x0 + cx0 + k;
        if (gy < H && gx < W) {
            pg[(size_t)gy * W + gx] = gacc[k] * p.scale;
            sl += (double)sacc[k];
        }
    }
    if (p.partials) {
        red[tid] = sl;
        __syncthreads();
        for (int st = G::NT / 2; st > 0; st >>= 1) {
            if (tid < st) red[tid] += red[tid + st];
            __syncthreads();
        }
        if (tid == 0)
            p.partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] =
                red[0] * (double)p.scale * (double)p.inv_sigma_r;
    }
}

template <int KIND, int RAD, int TH, int TW, int TWT>
cudaError_t launch_bwd(const BwdParams &prm, int count, cudaStream_t s) {
    using G = BwdGeom<KIND, RAD, TH, TW, TWT>;
    static_assert(G::SMEM <= 227 * 1024, "shared memory");
    static_assert((G::NT & (G::NT - 1)) == 0, "reduction needs a power-of-two block");
    auto kern = bf_tile_bwd<KIND, RAD, TH, TW, TWT>;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    dim3 grid((prm.W + TW - 1) / TW, (prm.H + TH - 1) / TH, count);
    kern<<<grid, G::NT, G::SMEM, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace bf

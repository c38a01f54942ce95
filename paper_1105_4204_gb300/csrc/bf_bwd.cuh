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

constexpr int kBwdTH = 32, kBwdTW = 64, kBwdTWT = 8;  // backward tile and segment

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
    static constexpr int SF = (EW + 3) / 4 * 4;
    // filtered planes as rows of float2 {cos part, sin part}; the row stride
    // covers the columns phase 1 writes and the float4s a segment reads, and
    // is 2 mod 4 float2 (an odd number of 16-byte units)
    static constexpr int LN2 = (LN + 1) / 2 * 2;
    static constexpr int SV2_MIN = (EW > TW - TWT + LN2 ? EW : TW - TWT + LN2);
    static constexpr int SV2 = (SV2_MIN + 3) / 4 * 4 + 2;
    static constexpr int SC2 = (TW + 3) / 4 * 4 + 2;
    static constexpr int NPL = 3;  // pair planes held at once
    static constexpr int T_FLOATS = EH * SF;  // one extended tile
    static constexpr int V_FLOATS = NPL * 2 * TH * SV2;
    static constexpr int C_FLOATS = 2 * TH * SC2;
    static constexpr size_t SMEM =
        sizeof(float) * (size_t)(3 * T_FLOATS + V_FLOATS + C_FLOATS) + sizeof(double) * NT;
    static_assert(TW % TWT == 0 && TWT % 4 == 0, "segments");
    static_assert(NT <= 1024, "block");
    static_assert(2 * EW <= NT, "one phase-1 item per thread");
};

// SIG: dL/dsigma_r requested.  Without it the f^2 planes, which only that
// derivative needs, are neither filtered nor combined.
template <int KIND, int RAD, int TH, int TW, int TWT, bool SIG>
__global__ void __launch_bounds__(BwdGeom<KIND, RAD, TH, TW, TWT>::NT)
    bf_tile_bwd(const __grid_constant__ BwdParams p) {
    using G = BwdGeom<KIND, RAD, TH, TW, TWT>;
    constexpr int HALO = G::HALO, EH = G::EH, EW = G::EW;
    constexpr int SV2 = G::SV2, SC2 = G::SC2;
    // round A's three planes in one sweep while the two pairs' filter window
    // fits in registers
    constexpr bool kOneSweep = KIND == 0 ? RAD <= 12 : RAD <= 4;
    extern __shared__ float4 smem4[];
    float *Fs = reinterpret_cast<float *>(smem4);  // f, clamp-extended
    float *As = Fs + G::T_FLOATS;                   // alpha, zero outside the image
    float *Os = As + G::T_FLOATS;                   // o, clamp-extended
    float *V = Os + G::T_FLOATS;                    // filtered pair planes (3 x TH x SV2 float2)
    float *CC = V + G::V_FLOATS;                    // {cos, sin} at the tile's pixels
    double *red = reinterpret_cast<double *>(CC + G::C_FLOATS);

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

    // phase-1 identity: (extended column j1, q1 = cos | sin); adjacent lanes
    // take cos and sin of one column, so their stores are contiguous
    const int j1 = tid >> 1;
    const int q1 = tid & 1;
    const bool p1 = tid < 2 * EW;
    const bool own_col = j1 >= HALO && j1 < HALO + TW;
    const float ph0 = q1 ? 0.f : 0.25f;  // cos(t) = sin(t + quarter turn)

    // one phase-2 pass: filter row pi of pair plane `pl` horizontally from
    // column cx0 and hand output k to use(k, z)
    auto hpass = [&](int pl, auto &&use) {
        const float4 *src4 =
            reinterpret_cast<const float4 *>(V + 2 * ((size_t)pl * TH * SV2 + pi * SV2 + cx0));
        float4 ld[(G::LN + 1) / 2];
        auto gen = [&](int i) {
            if ((i & 1) == 0) ld[i >> 1] = src4[i >> 1];
            const float4 v = ld[i >> 1];
            return (i & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
        };
        filt2_stream<KIND, RAD, G::LN>(gen, use, p.taps.w2);
    };

    const int n_terms = p.terms.n_terms;
    for (int m = 0; m < n_terms; ++m) {
        const float am = p.terms.a[m];
        const float tm = p.terms.t[m];
        const float wm = p.omega[m];
        // ================= round A: W of (c, s), (f c, f s), (f^2 c, f^2 s)
        __syncthreads();
        if (p1) {
            const float *fcol = Fs + j1;
            float *ccol = CC + 2 * (j1 - HALO) + q1;
            float *v0 = V + 2 * j1 + q1;
            auto gen_x = [&](int i, float &fv) {
                fv = fcol[i * G::SF];
                return sin_turns(fmaf(tm, fv, ph0));
            };
            if constexpr (!SIG) {
                // dL/df only: (x, f x)
                auto gen = [&](int i) {
                    float fv;
                    const float x = gen_x(i, fv);
                    if (i >= HALO && i < HALO + TH && own_col) ccol[(i - HALO) * 2 * SC2] = x;
                    return make_float2(x, x * fv);
                };
                auto sink = [&](int k, float2 y) {
                    v0[k * 2 * SV2] = y.x;
                    v0[(TH + k) * 2 * SV2] = y.y;
                };
                Ahead<kGenAhead, EH, decltype(gen)> ahead(gen);
                filt2_stream<KIND, RAD, EH>(ahead, sink, p.taps.w2);
            } else if constexpr (kOneSweep) {
                // (x, f x) and (f^2 x, 0) of one generated x in one sweep
                auto gen = [&](int i) {
                    float fv;
                    const float x = gen_x(i, fv);
                    if (i >= HALO && i < HALO + TH && own_col) ccol[(i - HALO) * 2 * SC2] = x;
                    Pairs<2> o;
                    const float fx = x * fv;
                    o.v[0] = make_float2(x, fx);
                    o.v[1] = make_float2(fx * fv, 0.f);
                    return o;
                };
                auto sink = [&](int k, const Pairs<2> &y) {
                    v0[k * 2 * SV2] = y.v[0].x;
                    v0[(TH + k) * 2 * SV2] = y.v[0].y;
                    v0[(2 * TH + k) * 2 * SV2] = y.v[1].x;
                };
                AheadN<kGenAhead, EH, 2, decltype(gen)> ahead(gen);
                filt2n_stream<KIND, RAD, EH, 2>(ahead, sink, p.taps.w2);
            } else {
                // wide supports: two sweeps, x generated again for the second
                auto gen = [&](int i) {
                    float fv;
                    const float x = gen_x(i, fv);
                    if (i >= HALO && i < HALO + TH && own_col) ccol[(i - HALO) * 2 * SC2] = x;
                    return make_float2(x, x * fv);
                };
                auto sink = [&](int k, float2 y) {
                    v0[k * 2 * SV2] = y.x;
                    v0[(TH + k) * 2 * SV2] = y.y;
                };
                Ahead<kGenAhead, EH, decltype(gen)> ahead(gen);
                filt2_stream<KIND, RAD, EH>(ahead, sink, p.taps.w2);
                auto gen2 = [&](int i) {
                    float fv;
                    const float x = gen_x(i, fv);
                    return make_float2(x * fv * fv, 0.f);
                };
                auto sink2 = [&](int k, float2 y) { v0[(2 * TH + k) * 2 * SV2] = y.x; };
                Ahead<kGenAhead, EH, decltype(gen2)> ahead2(gen2);
                filt2_stream<KIND, RAD, EH>(ahead2, sink2, p.taps.w2);
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
                const float2 cs = *reinterpret_cast<const float2 *>(CC + 2 * (pi * SC2 + cx0 + k));
                kc[k] = kk * cs.x;
                ks[k] = kk * cs.y;
                fp[k] = Fs[ti];
                op[k] = Os[ti];
            }
            // (W[c], W[s])
            hpass(0, [&](int k, float2 z) {
                gacc[k] = fmaf(ks[k] * op[k], z.x, fmaf(-kc[k] * op[k], z.y, gacc[k]));
                if constexpr (SIG)
                    sacc[k] = fmaf(-ks[k] * fp[k] * op[k], z.x,
                                   fmaf(kc[k] * fp[k] * op[k], z.y, sacc[k]));
            });
            // (W[f c], W[f s])
            hpass(1, [&](int k, float2 z) {
                gacc[k] = fmaf(-ks[k], z.x, fmaf(kc[k], z.y, gacc[k]));
                if constexpr (SIG) {
                    const float fo = fp[k] + op[k];
                    sacc[k] = fmaf(ks[k] * fo, z.x, fmaf(-kc[k] * fo, z.y, sacc[k]));
                }
            });
            // (W[f^2 c], W[f^2 s])
            if constexpr (SIG) {
                hpass(2, [&](int k, float2 z) {
                    sacc[k] = fmaf(-ks[k], z.x, fmaf(kc[k], z.y, sacc[k]));
                });
            }
        }
        // ================= round B: W^T of (alpha c, alpha s), (alpha o c, alpha o s)
        __syncthreads();
        if (p1) {
            const float *fcol = Fs + j1;
            const float *acol = As + j1;
            const float *ocol = Os + j1;
            float *v0 = V + 2 * j1 + q1;
            auto gen = [&](int i) {
                const float g = acol[i * G::SF] * sin_turns(fmaf(tm, fcol[i * G::SF], ph0));
                return make_float2(g, g * ocol[i * G::SF]);
            };
            auto sink = [&](int k, float2 y) {
                v0[k * 2 * SV2] = y.x;
                v0[(TH + k) * 2 * SV2] = y.y;
            };
            Ahead<kGenAhead, EH, decltype(gen)> ahead(gen);
            filt2_stream<KIND, RAD, EH>(ahead, sink, p.taps.w2);
            // tail fold at the image's first / last row (a one-row image
            // keeps the whole mass on its only row); values regenerated
            if (top >= 0 && bot == top) {
                const float2 g = gen(HALO);
                v0[top * 2 * SV2] = p.total * g.x;
                v0[(TH + top) * 2 * SV2] = p.total * g.y;
            } else if (top >= 0) {
                float2 acc = make_float2(0.f, 0.f);
                for (int d = 0; d <= HALO; ++d) {
                    const float2 g = gen(HALO + d);
                    acc.x = fmaf(p.tail[d], g.x, acc.x);
                    acc.y = fmaf(p.tail[d], g.y, acc.y);
                }
                v0[top * 2 * SV2] = acc.x;
                v0[(TH + top) * 2 * SV2] = acc.y;
            }
            if (bot >= 0 && bot != top) {
                // image row H-1-d sits at extended row bot + HALO - d (>= 0)
                float2 acc = make_float2(0.f, 0.f);
                for (int d = 0; d <= HALO; ++d) {
                    const float2 g = gen(bot + HALO - d);
                    acc.x = fmaf(p.tail[d], g.x, acc.x);
                    acc.y = fmaf(p.tail[d], g.y, acc.y);
                }
                v0[bot * 2 * SV2] = acc.x;
                v0[(TH + bot) * 2 * SV2] = acc.y;
            }
        }
        __syncthreads();
        {
            float ca[TWT], cb[TWT], cc[TWT], cd[TWT];
#pragma unroll
            for (int k = 0; k < TWT; ++k) {
                const int ti = (pi + HALO) * G::SF + cx0 + k + HALO;
                const float2 cs = *reinterpret_cast<const float2 *>(CC + 2 * (pi * SC2 + cx0 + k));
                const float c = cs.x, s = cs.y;
                const float fv = Fs[ti];
                const float aw = am * wm;
                ca[k] = am * c - aw * s * fv;  // W^T[alpha c]
                cb[k] = am * s + aw * c * fv;  // W^T[alpha s]
                cc[k] = aw * s;                // W^T[alpha o c]
                cd[k] = -aw * c;               // W^T[alpha o s]
            }
#pragma unroll 1
            for (int pl = 0; pl < 2; ++pl) {
                // tail fold at the image's first / last column: these outputs
                // take the folded sums instead of the filter's
                const float2 *row =
                    reinterpret_cast<const float2 *>(V) + (size_t)pl * TH * SV2 + pi * SV2;
                int kl = -1, kr = -1;
                float2 zl = make_float2(0.f, 0.f), zr = zl;
                if (lef >= 0 && rig == 0 && cx0 == 0) {
                    const float2 v = row[HALO];
                    zl = make_float2(p.total * v.x, p.total * v.y);
                    kl = 0;
                } else if (lef >= 0 && cx0 == 0) {
                    for (int d = 0; d <= HALO; ++d) {
                        const float2 v = row[HALO + d];
                        zl.x = fmaf(p.tail[d], v.x, zl.x);
                        zl.y = fmaf(p.tail[d], v.y, zl.y);
                    }
                    kl = 0;
                }
                if (rig >= cx0 && rig < cx0 + TWT && !(lef >= 0 && rig == 0)) {
                    for (int d = 0; d <= HALO; ++d) {
                        const float2 v = row[rig + HALO - d];
                        zr.x = fmaf(p.tail[d], v.x, zr.x);
                        zr.y = fmaf(p.tail[d], v.y, zr.y);
                    }
                    kr = rig - cx0;
                }
                hpass(pl, [&](int k, float2 z) {
                    if (k == kl) z = zl;
                    if (k == kr) z = zr;
                    const float c0 = pl == 0 ? ca[k] : cc[k];
                    const float c1 = pl == 0 ? cb[k] : cd[k];
                    gacc[k] = fmaf(c0, z.x, fmaf(c1, z.y, gacc[k]));
                });
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
    auto kern = prm.partials ? bf_tile_bwd<KIND, RAD, TH, TW, TWT, true>
                             : bf_tile_bwd<KIND, RAD, TH, TW, TWT, false>;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        for (auto k : {bf_tile_bwd<KIND, RAD, TH, TW, TWT, true>,
                       bf_tile_bwd<KIND, RAD, TH, TW, TWT, false>}) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)G::SMEM);
            if (e != cudaSuccess) return e;
        }
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    dim3 grid((prm.W + TW - 1) / TW, (prm.H + TH - 1) / TH, count);
    kern<<<grid, G::NT, G::SMEM, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace bf

// Adjoint (backward) of the filter for the 3-pass box with 8 < r <= 64, whose
// support does not fit the fused adjoint's tile.  The chain rule is the fused
// adjoint's (bf_bwd.cuh), evaluated one term at a time through planes in the
// library's device scratch:
//
//   round A: the clamp-extended planes c, s, f c, f s and, when dL/dsigma_r is
//            asked for, f^2 c, f^2 s, filtered by W (vertical, then
//            horizontal running sums of the three boxes), combined per pixel
//            into dL/df and the dL/dsigma_r sums;
//   round B: the zero-extended planes alpha c, alpha s, alpha o c, alpha o s
//            (alpha = u / Q, o the forward output) filtered by W^T, which per
//            axis is the zero-extended box with the tail mass folded back
//            onto the first and last pixel, W^T[g](0) = sum_p T(p) g(p),
//            T(p) = sum_{d >= p} w1(d) (a one-pixel axis keeps the whole
//            mass), combined per pixel into dL/df.
//
// Every polynomial factor of the planes and of the combine is a product of
// differences f(y) - f(x), f(y) - o(x), so f and o enter them shifted by the
// middle of the range, c0 = T / 2 (the phases keep f): the same gradient with
// planes of a quarter of the magnitude, which the long running sums need (the
// f^2 planes of an unnormalised box at r = 12 reach 10^9).  The boxes run
// unnormalised (integer-count taps); the common scale is applied to each
// term's contribution.  dL/df accumulates in the output over the
// terms, round A before round B, in term order; dL/dsigma_r in one double per
// 32 x 64 block, summed over the terms in order and reduced afterwards as the
// fused adjoint's partials are.  Every kernel reads and writes device memory:
// this path trades bandwidth for a support of any size.
//
// The recursive Gaussian (Section 3) runs the same rounds with its own line
// filter per axis in place of the boxes (rb_vpass, rb_hpass): W is the
// forward line, the causal recursion from the steady state of the first
// sample over the line and P samples of its last one, then the anticausal
// recursion from the steady state of the causal pass's last output.  W^T
// reverses those steps: the zero-extended line through the causal recursion
// from zero, the anticausal recursion from zero with the adjoint of the
// anticausal start added at the last sample, then the adjoint of the causal
// start added at the first pixel and the extension's samples folded onto the
// last pixel.  Both recursions run in the difference form of the forward
// filter (unit DC gain whatever the rounding of B); the extension's samples
// go to buffers of their own.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "bf_internal.h"
#include "bf_tile.cuh"

namespace bf {

namespace {

constexpr int kLbCols = 64;   // columns per vertical-pass block (a thread each)
constexpr int kLbRowsV = 32;  // output rows per vertical-pass block
constexpr int kLbRowsH = 64;  // rows per horizontal-pass block (a thread each)
constexpr int kLbColsH = 64;  // output columns per horizontal-pass block
constexpr int kLbMaxHalo = 3 * 64;
constexpr int kCombTH = 32, kCombTW = 64;  // combine block: the fused adjoint's partial grid
constexpr int kLbPlanes = 6;          // plane slots per image in each scratch buffer
constexpr size_t kLbChunkBytes = 1ull << 31;  // scratch for one chunk of a stack

struct LbParams {
    const float *f, *o, *q, *u;  // image 0 of the chunk; images n apart
    int H, W;
    int r, halo;         // box half-width, 3 r
    float tail[kLbMaxHalo + 1];  // T(d), integer counts, d = 0 .. halo
    float total;         // (2 r + 1)^3, the mass of one axis
    float scale;         // (2 r + 1)^-6, the 2-D normalisation
    float inv_sigma_r;
    float c0;            // shift of f and o in the polynomial factors
};

// Three unnormalised boxes of half-width r, in place on a[0 .. n_in) (stride
// apart); output k lands in a[k] for k < n_in - 6 r.  The running sums are
// compensated (Kahan): the adjoint combines nearly cancelling planes, so the
// sums' rounding must not grow along the sweep.
__device__ void box3_inplace(float *a, int stride, int n_in, int r) {
    int n = n_in;
    for (int pass = 0; pass < 3; ++pass) {
        const int nout = n - 2 * r;
        float s = 0.f, comp = 0.f;
        auto add = [&](float v) {
            const float y = __fsub_rn(v, comp);
            const float t = __fadd_rn(s, y);
            comp = __fsub_rn(__fsub_rn(t, s), y);
            s = t;
        };
        for (int d = 0; d <= 2 * r; ++d) add(a[d * stride]);
        float prev = a[0];
        a[0] = s;
        for (int k = 1; k < nout; ++k) {
            const float nxt = a[(k + 2 * r) * stride];
            const float cur = a[k * stride];
            add(nxt);
            add(-prev);
            a[k * stride] = s;
            prev = cur;
        }
        n = nout;
    }
}

// Plane q of a round at pixel (y, x) of the image (y, x inside it).
//   round A: 0 c, 1 s, 2 f~ c, 3 f~ s, 4 f~^2 c, 5 f~^2 s
//   round B: 0 alpha c, 1 alpha s, 2 alpha o~ c, 3 alpha o~ s
// (f~ = f - c0, o~ = o - c0; the phase of c and s is that of f)
template <int ROUND>
__device__ __forceinline__ float lb_plane(const LbParams &p, long long i, int q, float tm) {
    const float fv = __ldg(p.f + i);
    const float x = (q & 1) ? sin_turns(tm * fv) : sin_turns(fmaf(tm, fv, 0.25f));
    if constexpr (ROUND == 0) {
        if (q < 2) return x;
        const float ft = fv - p.c0;
        const float fx = x * ft;
        return q < 4 ? fx : fx * ft;
    } else {
        const float g = __ldg(p.u + i) / __ldg(p.q + i) * x;
        return q < 2 ? g : g * (__ldg(p.o + i) - p.c0);
    }
}

// Vertical pass: generates plane q of image img (blockIdx.z = img * planes +
// q) over the block's rows plus the halo (round A clamps the rows, round B is
// zero outside the image) and filters it; round B then folds the tails onto
// rows 0 and H - 1.  Plane q of image img is at (img * kLbPlanes + q) * n.
// grid: (ceil(W / kLbCols), ceil(H / kLbRowsV), images x planes); block: kLbCols
template <int ROUND>
__global__ void __launch_bounds__(kLbCols) lb_vpass(const __grid_constant__ LbParams p,
                                                   float *__restrict__ dst, float tm,
                                                   int planes) {
    extern __shared__ float lb_sm[];
    const int H = p.H, W = p.W, halo = p.halo;
    const long long n = (long long)H * W;
    const int x = blockIdx.x * kLbCols + threadIdx.x;
    const int y0 = blockIdx.y * kLbRowsV;
    const int img = blockIdx.z / planes, q = blockIdx.z - img * planes;
    const long long ioff = img * n;
    const int xc = min(x, W - 1);
    const int n_in = kLbRowsV + 2 * halo;
    float *a = lb_sm + threadIdx.x;
    // unrolled so that eight independent loads are in flight before their stores
#pragma unroll 8
    for (int i = 0; i < n_in; ++i) {
        const int gy = y0 - halo + i;
        float v;
        if constexpr (ROUND == 0) {
            v = lb_plane<0>(p, ioff + (long long)min(max(gy, 0), H - 1) * W + xc, q, tm);
        } else {
            v = (gy >= 0 && gy < H) ? lb_plane<1>(p, ioff + (long long)gy * W + xc, q, tm)
                                    : 0.f;
        }
        a[i * kLbCols] = v;
    }
    // round B: the tail folds of the image's first and last row, from the
    // unfiltered values (row y sits at staged index y - y0 + halo)
    float fold_top = 0.f, fold_bot = 0.f;
    const int bi = H - 1 - y0;  // output index of row H - 1 in this block
    const bool has_top = ROUND == 1 && y0 == 0;
    const bool has_bot = ROUND == 1 && bi >= 0 && bi < kLbRowsV && H > 1;
    if (has_top) {
        if (H == 1) {
            fold_top = p.total * a[halo * kLbCols];
        } else {
            for (int d = 0; d <= halo; ++d)
                fold_top = fmaf(p.tail[d], a[(halo + d) * kLbCols], fold_top);
        }
    }
    if (has_bot)
        for (int d = 0; d <= halo; ++d)
            fold_bot = fmaf(p.tail[d], a[(bi + halo - d) * kLbCols], fold_bot);
    box3_inplace(a, kLbCols, n_in, p.r);
    if (x >= W) return;
    float *out = dst + (img * kLbPlanes + q) * n;
    for (int i = 0; i < kLbRowsV && y0 + i < H; ++i) {
        float v = a[i * kLbCols];
        if (has_top && i == 0) v = fold_top;
        if (has_bot && i == bi) v = fold_bot;
        out[(long long)(y0 + i) * W + x] = v;
    }
}

// Horizontal pass of plane q of image img (blockIdx.z = img * planes + q):
// round A clamps the columns, round B is zero outside the image and folds the
// tails onto columns 0 and W - 1.
// grid: (ceil(W / kLbColsH), ceil(H / kLbRowsH), images x planes); block: kLbRowsH
template <int ROUND>
__global__ void __launch_bounds__(kLbRowsH) lb_hpass(const __grid_constant__ LbParams p,
                                                    const float *__restrict__ src,
                                                    float *__restrict__ dst, int planes) {
    extern __shared__ float lb_sm[];
    const int H = p.H, W = p.W, halo = p.halo;
    const long long n = (long long)H * W;
    const int x0 = blockIdx.x * kLbColsH;
    const int y0 = blockIdx.y * kLbRowsH;
    const int img = blockIdx.z / planes, q = blockIdx.z - img * planes;
    const float *s = src + (img * kLbPlanes + q) * n;
    float *d_out = dst + (img * kLbPlanes + q) * n;
    const int n_in = kLbColsH + 2 * halo;
    const int stride = n_in | 1;  // odd: a thread per row hits distinct banks
    // the staged rows x columns as asynchronous 4-byte copies (the warp does
    // not wait for each load): round A from the clamped column, round B with
    // a zero fill outside the image
    for (int idx = threadIdx.x; idx < kLbRowsH * n_in; idx += kLbRowsH) {
        const int rr = idx / n_in, j = idx - (idx / n_in) * n_in;
        const int gy = min(y0 + rr, H - 1);
        const int gx = x0 - halo + j;
        const bool in = gx >= 0 && gx < W;
        const float *src_el = s + (long long)gy * W + min(max(gx, 0), W - 1);
        const unsigned dst = (unsigned)__cvta_generic_to_shared(lb_sm + rr * stride + j);
        const int bytes = (ROUND == 0 || in) ? 4 : 0;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src_el),
                     "r"(bytes)
                     : "memory");
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    float *a = lb_sm + threadIdx.x * stride;
    float fold_l = 0.f, fold_r = 0.f;
    const int bj = W - 1 - x0;  // output index of column W - 1 in this block
    const bool has_l = ROUND == 1 && x0 == 0;
    const bool has_r = ROUND == 1 && bj >= 0 && bj < kLbColsH && W > 1;
    if (has_l) {
        if (W == 1) {
            fold_l = p.total * a[halo];
        } else {
            for (int d = 0; d <= halo; ++d) fold_l = fmaf(p.tail[d], a[halo + d], fold_l);
        }
    }
    if (has_r)
        for (int d = 0; d <= halo; ++d) fold_r = fmaf(p.tail[d], a[bj + halo - d], fold_r);
    box3_inplace(a, 1, n_in, p.r);
    if (has_l) a[0] = fold_l;
    if (has_r) a[bj] = fold_r;
    __syncthreads();
#pragma unroll 8
    for (int idx = threadIdx.x; idx < kLbRowsH * kLbColsH; idx += kLbRowsH) {
        const int rr = idx / kLbColsH, j = idx - (idx / kLbColsH) * kLbColsH;
        const int gy = y0 + rr;
        if (gy < H && x0 + j < W) d_out[(long long)gy * W + x0 + j] = lb_sm[rr * stride + j];
    }
}

// Per-pixel combine of one term's filtered planes of image blockIdx.z (as
// the fused adjoint combines them), added to its grad (round A of the first
// term writes it); round A with SIG also adds this block's dL/dsigma_r sum to
// its partial.
// grid: (ceil(W / kCombTW), ceil(H / kCombTH), images); block: 256
template <int ROUND, bool SIG>
__global__ void __launch_bounds__(256) lb_combine(const __grid_constant__ LbParams p,
                                                 const float *__restrict__ A_all,
                                                 float *__restrict__ grad_all,
                                                 double *__restrict__ partials_all, float am,
                                                 float tm, float wm, int first) {
    __shared__ double red[256];
    const int H = p.H, W = p.W;
    const long long n = (long long)H * W;
    const int img = blockIdx.z;
    const float *A = A_all + (long long)img * kLbPlanes * n;
    float *grad = grad_all + img * n;
    const long long ioff = img * n;
    const int x = blockIdx.x * kCombTW + threadIdx.x % kCombTW;
    double sl = 0.0;
#pragma unroll
    for (int k = 0; k < kCombTH * kCombTW / 256; ++k) {
        const int y = blockIdx.y * kCombTH + threadIdx.x / kCombTW + k * (256 / kCombTW);
        if (y >= H || x >= W) continue;
        const long long i = (long long)y * W + x;
        const float f0 = __ldg(p.f + ioff + i);
        const float fv = f0 - p.c0, ov = __ldg(p.o + ioff + i) - p.c0;  // shifted
        const float al = __ldg(p.u + ioff + i) / __ldg(p.q + ioff + i);
        const float c = sin_turns(fmaf(tm, f0, 0.25f)), s = sin_turns(tm * f0);
        float g = 0.f;
        if constexpr (ROUND == 0) {
            const float kk = am * wm * al;
            const float kc = kk * c, ks = kk * s;
            const float wc = A[i], ws = A[n + i], wfc = A[2 * n + i], wfs = A[3 * n + i];
            g = fmaf(ks * ov, wc, fmaf(-kc * ov, ws, g));
            g = fmaf(-ks, wfc, fmaf(kc, wfs, g));
            if constexpr (SIG) {
                float sa = 0.f;
                sa = fmaf(-ks * fv * ov, wc, fmaf(kc * fv * ov, ws, sa));
                const float fo = fv + ov;
                sa = fmaf(ks * fo, wfc, fmaf(-kc * fo, wfs, sa));
                sa = fmaf(-ks, A[4 * n + i], fmaf(kc, A[5 * n + i], sa));
                sl += (double)sa;
            }
        } else {
            const float aw = am * wm;
            const float ca = am * c - aw * s * fv;  // W^T[alpha c]
            const float cb = am * s + aw * c * fv;  // W^T[alpha s]
            const float cc = aw * s;                // W^T[alpha o c]
            const float cd = -aw * c;               // W^T[alpha o s]
            g = fmaf(ca, A[i], fmaf(cb, A[n + i], g));
            g = fmaf(cc, A[2 * n + i], fmaf(cd, A[3 * n + i], g));
        }
        const float add = g * p.scale;
        grad[i] = first ? add : grad[i] + add;
    }
    if constexpr (ROUND == 0 && SIG) {
        red[threadIdx.x] = sl;
        __syncthreads();
        for (int st = 128; st > 0; st >>= 1) {
            if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            double *partials = partials_all + (size_t)img * gridDim.x * gridDim.y;
            const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
            const double v = red[0] * (double)p.scale * (double)p.inv_sigma_r;
            partials[b] = first ? v : partials[b] + v;
        }
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---- recursive Gaussian -------------------------------------------------------

constexpr int kRbThreads = 64;  // lines per block (a thread each)

struct RbCoef {
    float B;          // the recursions' input weight
    float D1, D2;     // a2 + a3 and a3 of the difference form
    float oneMinusB;  // a1 + a2 + a3, the weight of a steady start's three samples
    float invB;
    int P;            // extension past the last sample
};

// One step of the difference form: w(e) = w(e-1) + [B (x - w(e-1)) - (D1 d1 + D2 d2)],
// d1, d2 the last two increments (the recursion B x + a1 w(e-1) + a2 w(e-2) + a3 w(e-3)).
__device__ __forceinline__ float rb_step(const RbCoef &c, float x, float &w, float &d1,
                                         float &d2) {
    const float dw = __fsub_rn(__fmul_rn(c.B, __fsub_rn(x, w)),
                               __fmaf_rn(c.D2, d2, __fmul_rn(c.D1, d1)));
    w = __fadd_rn(w, dw);
    d2 = d1;
    d1 = dw;
    return w;
}

// The line filter (ROUND 0: W; 1: W^T) of one line of n samples, stride st
// apart in `line` (samples 0 .. n-1, filtered in place) and `ext` (the P
// extension samples, stride st), whose input sample k < n comes from in(k).
template <int ROUND, class In>
__device__ __forceinline__ void rb_line(const RbCoef &c, In &&in, int n, float *line,
                                        float *ext, long long st) {
    constexpr int CH = 8;  // samples whose loads are issued together
    const int E = n + c.P;
    float w, d1 = 0.f, d2 = 0.f;
    float z1 = 0.f, z2 = 0.f, z3 = 0.f;  // the causal pass's last three outputs
    // ROUND 0: the steady state of the first sample, and the extension's value
    const float first_in = ROUND == 0 ? in(0) : 0.f;
    const float last_in = ROUND == 0 ? in(n - 1) : 0.f;
    w = first_in;
    for (int k0 = 0; k0 < E; k0 += CH) {
        float xs[CH];
#pragma unroll
        for (int d = 0; d < CH; ++d) {
            const int k = k0 + d;
            xs[d] = k < n ? in(k) : last_in;  // ROUND 1: last_in is 0 (zero extension)
        }
#pragma unroll
        for (int d = 0; d < CH; ++d) {
            const int k = k0 + d;
            if (k < E) {
                rb_step(c, xs[d], w, d1, d2);
                if (k < n) line[k * st] = w;
                else ext[(k - n) * st] = w;
                z3 = z2;
                z2 = z1;
                z1 = w;
            }
        }
    }
    // anticausal: ROUND 0 from the steady state of the causal pass's last
    // output; ROUND 1 from zero, the adjoint of that start entering at E - 1
    if constexpr (ROUND == 0) {
        w = z1;
    } else {
        w = 0.f;
    }
    d1 = d2 = 0.f;
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, fold = 0.f;
    for (int k1 = E - 1; k1 >= 0; k1 -= CH) {
        float xs[CH];
#pragma unroll
        for (int d = 0; d < CH; ++d) {
            const int k = k1 - d;
            xs[d] = k >= 0 ? (k < n ? line[k * st] : ext[(k - n) * st]) : 0.f;
        }
#pragma unroll
        for (int d = 0; d < CH; ++d) {
            const int k = k1 - d;
            if (k >= 0) {
                float x = xs[d];
                if (ROUND == 1 && k == E - 1)
                    x = __fadd_rn(x, __fmul_rn(__fmaf_rn(c.oneMinusB, z1,
                                                         __fmaf_rn(c.D1, z2, __fmul_rn(c.D2, z3))),
                                               c.invB));
                rb_step(c, x, w, d1, d2);
                if (k < n) line[k * st] = w;
                else if (ROUND == 1) fold = __fadd_rn(fold, w);
                v2 = v1;
                v1 = v0;
                v0 = w;
            }
        }
    }
    if constexpr (ROUND == 1) {
        // the causal start's adjoint on the first pixel, the extension folded
        // onto the last
        float first = __fadd_rn(v0, __fmul_rn(__fmaf_rn(c.oneMinusB, v0,
                                                        __fmaf_rn(c.D1, v1, __fmul_rn(c.D2, v2))),
                                              c.invB));
        if (n == 1) {
            first = __fadd_rn(first, fold);
        } else {
            line[(n - 1) * st] = __fadd_rn(line[(n - 1) * st], fold);
        }
        line[0] = first;
    }
}

// Vertical pass of plane q of image img (blockIdx.z = img * planes + q): the
// plane generated down each column (round A: every row of the image, round
// B: alpha-weighted) and filtered in place in dst; the extension rows in X
// (P rows per plane).
// grid: (ceil(W / kRbThreads), 1, images x planes); block: kRbThreads
template <int ROUND>
__global__ void __launch_bounds__(kRbThreads) rb_vpass(const __grid_constant__ LbParams p,
                                                      const RbCoef c, float *__restrict__ dst,
                                                      float *__restrict__ X, float tm,
                                                      int planes) {
    const int H = p.H, W = p.W;
    const long long n = (long long)H * W;
    const int x = blockIdx.x * kRbThreads + threadIdx.x;
    const int img = blockIdx.z / planes, q = blockIdx.z - img * planes;
    if (x >= W) return;
    const long long ioff = img * n + x;
    const long long pl = (long long)img * kLbPlanes + q;
    auto in = [&](int k) { return lb_plane<ROUND>(p, ioff + (long long)k * W, q, tm); };
    rb_line<ROUND>(c, in, H, dst + pl * n + x, X + pl * c.P * W + x, W);
}

// Horizontal pass of plane q of image img: src's rows filtered into dst; the
// extension columns in X (P per row).
// grid: (ceil(H / kRbThreads), 1, images x planes); block: kRbThreads
template <int ROUND>
__global__ void __launch_bounds__(kRbThreads) rb_hpass(const __grid_constant__ LbParams p,
                                                      const RbCoef c,
                                                      const float *__restrict__ src,
                                                      float *__restrict__ dst,
                                                      float *__restrict__ X, int planes) {
    const int H = p.H, W = p.W;
    const long long n = (long long)H * W;
    const int y = blockIdx.x * kRbThreads + threadIdx.x;
    const int img = blockIdx.z / planes, q = blockIdx.z - img * planes;
    if (y >= H) return;
    const long long pl = (long long)img * kLbPlanes + q;
    const float *row = src + pl * n + (long long)y * W;
    auto in = [&](int k) { return row[k]; };
    rb_line<ROUND>(c, in, W, dst + pl * n + (long long)y * W,
                   X + (pl * H + y) * (long long)c.P, 1);
}

}  // namespace

bool bwd_large_supported(const bf_plan *p) {
    if (p->kind == BF_SPATIAL_GAUSS_RECURSIVE) return p->rg_P >= 1;
    return p->kind == BF_SPATIAL_BOX_ITER && p->passes == 3 && p->r_box > 8 &&
           3 * p->r_box <= kLbMaxHalo;
}

// Extension samples per image of the recursive Gaussian's passes (P rows of
// W and H rows of P per plane); none for the box.
static size_t lb_ext(const bf_plan *pl, int H, int W) {
    if (pl->kind != BF_SPATIAL_GAUSS_RECURSIVE) return 0;
    return (size_t)kLbPlanes * (size_t)pl->rg_P * ((size_t)W + (size_t)H);
}

// Images of a stack per chunk: as many as kLbChunkBytes of scratch hold (at
// least one), and at most 65535 / kLbPlanes (the grid's z dimension).
static int lb_chunk(const bf_plan *pl, int H, int W, int count) {
    const size_t per =
        (2 * (size_t)kLbPlanes * (size_t)H * (size_t)W + lb_ext(pl, H, W)) * sizeof(float);
    const size_t fit = std::max<size_t>(1, kLbChunkBytes / per);
    return (int)std::min<size_t>(std::min<size_t>(fit, (size_t)count), 65535 / kLbPlanes);
}

// The recursive Gaussian's extension buffers for a chunk of k images: the
// vertical pass's P rows of W and the horizontal pass's H rows of P per plane.
static size_t lb_ext_v(const bf_plan *pl, int W, size_t k) {
    return pl->kind == BF_SPATIAL_GAUSS_RECURSIVE
               ? align256((size_t)kLbPlanes * pl->rg_P * (size_t)W * k * sizeof(float))
               : 0;
}
static size_t lb_ext_h(const bf_plan *pl, int H, size_t k) {
    return pl->kind == BF_SPATIAL_GAUSS_RECURSIVE
               ? align256((size_t)kLbPlanes * pl->rg_P * (size_t)H * k * sizeof(float))
               : 0;
}

size_t bwd_large_workspace(const bf_plan *pl, int H, int W, int count) {
    const size_t k = (size_t)lb_chunk(pl, H, W, count);
    const size_t n = (size_t)H * (size_t)W * k;
    return 2 * align256((size_t)kLbPlanes * n * sizeof(float)) + lb_ext_v(pl, W, k) +
           lb_ext_h(pl, H, k) + 256;
}

// count images n = H W apart; partials: count x ceil(W/64) x ceil(H/32)
// doubles (image k's at k x that), or nullptr without dL/dsigma_r.
cudaError_t launch_backward_large(const bf_plan *pl, const float *f, const float *o,
                                  const float *q, const float *u, float *grad,
                                  double *partials, int H, int W, int count, void *ws,
                                  cudaStream_t s) {
    const long long n = (long long)H * W;
    const int chunk = lb_chunk(pl, H, W, count);
    char *base = reinterpret_cast<char *>(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    const size_t buf = align256((size_t)kLbPlanes * n * chunk * sizeof(float));
    float *B = reinterpret_cast<float *>(base);  // vertical-pass planes
    float *A = reinterpret_cast<float *>(base + buf);
    LbParams p;
    p.H = H;
    p.W = W;
    p.inv_sigma_r = pl->sigma_r > 0 ? (float)(1.0 / pl->sigma_r) : 0.f;
    p.c0 = (float)(0.5 * pl->T);
    if (pl->kind == BF_SPATIAL_GAUSS_RECURSIVE) {
        // the recursive Gaussian: extension buffers after the two plane buffers
        float *XV = reinterpret_cast<float *>(base + 2 * buf);
        float *XH = reinterpret_cast<float *>(base + 2 * buf + lb_ext_v(pl, W, chunk));
        RbCoef c;
        c.B = (float)pl->rg[0];
        c.D1 = (float)(pl->rg[2] + pl->rg[3]);
        c.D2 = (float)pl->rg[3];
        c.oneMinusB = (float)(pl->rg[1] + pl->rg[2] + pl->rg[3]);
        c.invB = (float)(1.0 / pl->rg[0]);
        c.P = pl->rg_P;
        p.r = 0;
        p.halo = 0;
        p.total = 1.f;
        p.scale = 1.f;  // the recursive filter has unit gain
        for (int d = 0; d <= kLbMaxHalo; ++d) p.tail[d] = 0.f;
        const bool sig = partials != nullptr;
        const int planes_a = sig ? 6 : 4;
        const int gvx = (W + kRbThreads - 1) / kRbThreads, ghx = (H + kRbThreads - 1) / kRbThreads;
        const dim3 gc((W + kCombTW - 1) / kCombTW, (H + kCombTH - 1) / kCombTH);
        const size_t nblk = (size_t)gc.x * gc.y;
        const int nt = (int)pl->a32.size();
        for (int img0 = 0; img0 < count; img0 += chunk) {
            const int nimg = std::min(chunk, count - img0);
            p.f = f + img0 * n;
            p.o = o + img0 * n;
            p.q = q + img0 * n;
            p.u = u + img0 * n;
            float *g = grad + img0 * n;
            double *part = sig ? partials + img0 * nblk : nullptr;
            const dim3 gcz(gc.x, gc.y, nimg);
            for (int m = 0; m < nt; ++m) {
                const float am = pl->a32[m], tm = pl->turns32[m], wm = (float)pl->omega[m];
                rb_vpass<0><<<dim3(gvx, 1, nimg * planes_a), kRbThreads, 0, s>>>(p, c, B, XV, tm,
                                                                                  planes_a);
                rb_hpass<0><<<dim3(ghx, 1, nimg * planes_a), kRbThreads, 0, s>>>(p, c, B, A, XH,
                                                                                  planes_a);
                if (sig)
                    lb_combine<0, true><<<gcz, 256, 0, s>>>(p, A, g, part, am, tm, wm, m == 0);
                else
                    lb_combine<0, false><<<gcz, 256, 0, s>>>(p, A, g, nullptr, am, tm, wm,
                                                             m == 0);
                rb_vpass<1><<<dim3(gvx, 1, nimg * 4), kRbThreads, 0, s>>>(p, c, B, XV, tm, 4);
                rb_hpass<1><<<dim3(ghx, 1, nimg * 4), kRbThreads, 0, s>>>(p, c, B, A, XH, 4);
                lb_combine<1, false><<<gcz, 256, 0, s>>>(p, A, g, nullptr, am, tm, wm, 0);
                cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) return e;
            }
        }
        return cudaSuccess;
    }
    p.r = pl->r_box;
    p.halo = 3 * pl->r_box;
    const double L = 2.0 * pl->r_box + 1.0;
    const double norm = L * L * L;
    for (int d = 0; d <= kLbMaxHalo; ++d) p.tail[d] = 0.f;
    double t = 0.0;
    for (int d = p.halo; d >= 0; --d) {
        t += std::round(pl->w1[p.halo + d] * norm);  // integer counts of the 3-box taps
        p.tail[d] = (float)t;
    }
    p.total = (float)norm;
    p.scale = pl->q_scale;
    p.inv_sigma_r = pl->sigma_r > 0 ? (float)(1.0 / pl->sigma_r) : 0.f;
    p.c0 = (float)(0.5 * pl->T);
    const size_t smv = sizeof(float) * (size_t)(kLbRowsV + 2 * p.halo) * kLbCols;
    const size_t smh = sizeof(float) * (size_t)kLbRowsH * ((kLbColsH + 2 * p.halo) | 1);
    if (smv > 227 * 1024 || smh > 227 * 1024) return cudaErrorInvalidValue;
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        for (const void *k : {(const void *)lb_vpass<0>, (const void *)lb_vpass<1>,
                              (const void *)lb_hpass<0>, (const void *)lb_hpass<1>}) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     227 * 1024);
            if (e != cudaSuccess) return e;
        }
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    const bool sig = partials != nullptr;
    const int planes_a = sig ? 6 : 4;
    const dim3 gv((W + kLbCols - 1) / kLbCols, (H + kLbRowsV - 1) / kLbRowsV);
    const dim3 gh((W + kLbColsH - 1) / kLbColsH, (H + kLbRowsH - 1) / kLbRowsH);
    const dim3 gc((W + kCombTW - 1) / kCombTW, (H + kCombTH - 1) / kCombTH);
    const size_t nblk = (size_t)gc.x * gc.y;
    const int nt = (int)pl->a32.size();
    for (int img0 = 0; img0 < count; img0 += chunk) {
        const int nimg = std::min(chunk, count - img0);
        p.f = f + img0 * n;
        p.o = o + img0 * n;
        p.q = q + img0 * n;
        p.u = u + img0 * n;
        float *g = grad + img0 * n;
        double *part = sig ? partials + img0 * nblk : nullptr;
        const dim3 gcz(gc.x, gc.y, nimg);
        for (int m = 0; m < nt; ++m) {
            const float am = pl->a32[m], tm = pl->turns32[m], wm = (float)pl->omega[m];
            // round A: W of the clamp-extended planes
            lb_vpass<0><<<dim3(gv.x, gv.y, nimg * planes_a), kLbCols, smv, s>>>(p, B, tm,
                                                                               planes_a);
            lb_hpass<0><<<dim3(gh.x, gh.y, nimg * planes_a), kLbRowsH, smh, s>>>(p, B, A,
                                                                                planes_a);
            if (sig)
                lb_combine<0, true><<<gcz, 256, 0, s>>>(p, A, g, part, am, tm, wm, m == 0);
            else
                lb_combine<0, false><<<gcz, 256, 0, s>>>(p, A, g, nullptr, am, tm, wm, m == 0);
            // round B: W^T of the zero-extended planes
            lb_vpass<1><<<dim3(gv.x, gv.y, nimg * 4), kLbCols, smv, s>>>(p, B, tm, 4);
            lb_hpass<1><<<dim3(gh.x, gh.y, nimg * 4), kLbRowsH, smh, s>>>(p, B, A, 4);
            lb_combine<1, false><<<gcz, 256, 0, s>>>(p, A, g, nullptr, am, tm, wm, 0);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

}  // namespace bf

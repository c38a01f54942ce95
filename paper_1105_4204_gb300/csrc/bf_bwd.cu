// Instantiations and host side of the fused backward kernel, plus the
// deterministic reduction of the per-block dL/dsigma_r partials.
#include <cmath>

#include "bf_bwd.cuh"

namespace bf {

// Box instantiations live in bf_bwd_box.cu (compiled in parallel).
cudaError_t launch_bwd_box(int r, const BwdParams &prm, int count, cudaStream_t s);

namespace {


// One block sums the partials in a fixed order (per-thread strided sums, then
// a tree), so repeated runs give the same bits.
__global__ void bwd_reduce(const double *__restrict__ partials, int n, double *__restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s += partials[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

const int kGaussBwdRadii[] = {2, 4, 6, 9, 12, 18, 24};

int gauss_bwd_radius(int R) {
    for (int r : kGaussBwdRadii)
        if (r >= R) return r;
    return -1;
}

}  // namespace

bool bwd_supported(const bf_plan *p) {
    if (p->kind == BF_SPATIAL_GAUSS_TRUNC) return gauss_bwd_radius(p->R) > 0;
    return p->r_box >= 1 && p->r_box <= 8;
}

size_t bwd_blocks(int H, int W) {
    return (size_t)((W + kBwdTW - 1) / kBwdTW) * (size_t)((H + kBwdTH - 1) / kBwdTH);
}

cudaError_t launch_backward(const bf_plan *pl, const float *f, const float *o, const float *q,
                            const float *u, float *grad, double *grad_sigma_r, double *partials,
                            int H, int W, cudaStream_t s, int count) {
    BwdParams prm;
    prm.img_stride = (long long)H * W;
    prm.f = f;
    prm.o = o;
    prm.q = q;
    prm.u = u;
    prm.grad = grad;
    prm.partials = grad_sigma_r ? partials : nullptr;
    prm.H = H;
    prm.W = W;
    prm.inv_sigma_r = (float)(1.0 / pl->sigma_r);
    fill_terms(pl, &prm.terms);
    for (int k = 0; k < prm.terms.n_terms; ++k) prm.omega[k] = (float)pl->omega[k];
    for (int k = 0; k < 2 * BF_MAX_TAPS_R + 1; ++k) prm.taps.w[k] = 0.f;
    for (int k = 0; k < 2 * BF_MAX_TAPS_R + 1; ++k) prm.tail[k] = 0.f;
    if (pl->kind == BF_SPATIAL_GAUSS_TRUNC) {
        const int Ri = gauss_bwd_radius(pl->R);
        for (int k = 0; k < 2 * pl->R + 1; ++k) prm.taps.w[k + Ri - pl->R] = pl->w1f[k];
        // T(d) = sum_{e >= d} w1(e), d = 0 .. R
        double t = 0.0;
        for (int d = pl->R; d >= 0; --d) {
            t += pl->w1[pl->R + d];
            prm.tail[d] = (float)t;
        }
        prm.scale = 1.f;
        prm.total = 1.f;
    } else {
        // box: unnormalised integer-count taps, normalisation applied at the end
        const int r = pl->r_box;
        const double L = 2.0 * r + 1.0;
        const double norm = L * L * L;
        double t = 0.0;
        for (int d = 3 * r; d >= 0; --d) {
            t += std::round(pl->w1[3 * r + d] * norm);
            prm.tail[d] = (float)t;
        }
        prm.scale = pl->q_scale;
        prm.total = (float)norm;
    }
    pair_taps(&prm.taps);
    cudaError_t e;
    if (pl->kind == BF_SPATIAL_GAUSS_TRUNC) {
        switch (gauss_bwd_radius(pl->R)) {
            case 2: e = launch_bwd<0, 2, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s); break;
            case 4: e = launch_bwd<0, 4, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s); break;
            case 6: e = launch_bwd<0, 6, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s); break;
            case 9: e = launch_bwd<0, 9, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s); break;
            case 12: e = launch_bwd<0, 12, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s); break;
            case 18: e = launch_bwd<0, 18, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s); break;
            case 24: e = launch_bwd<0, 24, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s); break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        e = launch_bwd_box(pl->r_box, prm, count, s);
    }
    if (e != cudaSuccess) return e;
    if (grad_sigma_r) {
        bwd_reduce<<<1, 256, 0, s>>>(partials, (int)(bwd_blocks(H, W) * count), grad_sigma_r);
        e = cudaGetLastError();
    }
    return e;
}

// The fixed-order reduction of n partials into *out (used by the large-radius
// adjoint too).
cudaError_t launch_bwd_reduce(const double *partials, int n, double *out, cudaStream_t s) {
    bwd_reduce<<<1, 256, 0, s>>>(partials, n, out);
    return cudaGetLastError();
}

// Single-image form.
cudaError_t launch_backward(const bf_plan *pl, const float *f, const float *o, const float *q,
                            const float *u, float *grad, double *grad_sigma_r, double *partials,
                            int H, int W, cudaStream_t s) {
    return launch_backward(pl, f, o, q, u, grad, grad_sigma_r, partials, H, W, s, 1);
}

}  // namespace bf

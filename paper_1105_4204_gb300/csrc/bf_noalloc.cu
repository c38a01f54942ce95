// Backward pass for callers that cannot allocate device memory.
//
// bf_backward needs a small device scratch buffer for the per-block partial
// sums of dL/dsigma_r, which its caller allocates.  Some callers cannot:
// code running where a device allocation would synchronise or is forbidden
// (inside a real-time loop, under a memory pool that must not grow, in a
// plug-in host that owns all allocations).  bf_backward_noalloc keeps those
// partials in a fixed array that is part of the library image instead, so the
// call itself allocates nothing.
//
// In host code the array's name is only a host-side handle, not a device
// address: the first call on each device asks the runtime for the array's
// device address (cudaGetSymbolAddress, with that device current) and caches
// it; kernels are given that address.
#include <mutex>
#include <string>

#include "bf_internal.h"

namespace bf {
bool bwd_supported(const bf_plan *p);
size_t bwd_blocks(int H, int W);
cudaError_t launch_backward(const bf_plan *pl, const float *f, const float *o, const float *q,
                            const float *u, float *grad, double *grad_sigma_r, double *partials,
                            int H, int W, cudaStream_t s);
}  // namespace bf

// One double per backward block (a block covers 32 x 64 pixels): 16384
// partials, 128 KiB, resident on every device that loads the library until
// the process exits.
static constexpr int kStaticPartials = 16384;
static __device__ __align__(256) double g_bwd_partials[kStaticPartials];

namespace {

std::mutex g_mu;
double *g_dev_ptr[64];
bool g_ready[64];

}  // namespace

using namespace bf;

extern "C" bf_status bf_backward_noalloc(const bf_plan *plan, const float *f, const float *out,
                                         const float *q, const float *grad_out, float *grad_in,
                                         double *grad_sigma_r, int H, int W,
                                         cudaStream_t stream) {
    if (!plan) return fail(BF_EINVAL, "bf_backward_noalloc: plan is NULL");
    if (!f || !out || !q || !grad_out || !grad_in)
        return fail(BF_EINVAL, "bf_backward_noalloc: a data pointer is NULL");
    if (H < 1 || W < 1) return fail(BF_EINVAL, "bf_backward_noalloc: H and W must be >= 1");
    if ((long long)H * W > (1LL << 31) / 4)
        return fail(BF_EUNSUPPORTED, "bf_backward_noalloc: image too large");
    if (H > BF_MAX_ROWS)
        return fail(BF_EUNSUPPORTED, "bf_backward_noalloc: image taller than " +
                                         std::to_string(BF_MAX_ROWS) + " rows");
    if (!bwd_supported(plan))
        return fail(BF_EUNSUPPORTED, "bf_backward_noalloc: no kernel for this spatial support "
                                     "without device scratch (Gaussian R <= 24 or box r <= 8; "
                                     "the box with r > 8 and the recursive Gaussian run "
                                     "through scratch that bf_backward allocates)");
    if (grad_sigma_r && plan->cosine)
        return fail(BF_EINVAL, "bf_backward_noalloc: a cosine-polynomial plan has no sigma_r; "
                               "pass grad_sigma_r = NULL");
    double *partials = nullptr;
    if (grad_sigma_r) {
        const size_t need = bwd_blocks(H, W);
        if (need > (size_t)kStaticPartials)
            return fail(BF_EUNSUPPORTED,
                        "bf_backward_noalloc: image needs " + std::to_string(need) +
                            " partial sums of dL/dsigma_r, more than the fixed " +
                            std::to_string(kStaticPartials) +
                            " (ceil(W/64) * ceil(H/32) must be <= 16384); use bf_backward "
                            "with a workspace");
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_check(e, "bf_backward_noalloc: cudaGetDevice");
        if (dev < 0 || dev >= 64)
            return fail(BF_EUNSUPPORTED, "bf_backward_noalloc: device index above 63");
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_ready[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_bwd_partials);
            if (e != cudaSuccess)
                return cuda_check(e, "bf_backward_noalloc: cudaGetSymbolAddress");
            g_dev_ptr[dev] = static_cast<double *>(ptr);
            g_ready[dev] = true;
        }
        partials = g_dev_ptr[dev];
    }
    return cuda_check(launch_backward(plan, f, out, q, grad_out, grad_in, grad_sigma_r, partials,
                                      H, W, stream),
                      "bf_backward_noalloc launch");
}

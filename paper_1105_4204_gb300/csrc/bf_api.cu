// C-ABI entry points of libbf: argument checks, kernel selection, error text.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "bf_internal.h"

namespace bf {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

bf_status fail(bf_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

bf_status cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return BF_OK;
    return fail(BF_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                              cudaGetErrorString(e) + ")");
}

int gauss_tile_radius(int R);
int gauss_tile_shape_ids(int R, int *ids);
int box_tile_max_r();
int box_tile_shape_ids(int r, int *ids);
cudaError_t launch_tile_gauss(const bf_plan *pl, const BfImage &img, cudaStream_t s, int shape,
                              int split);
cudaError_t launch_tile_box(const bf_plan *pl, const BfImage &img, cudaStream_t s, int shape,
                            int split);

// Tile configurations picked by bf_forward_tune, per (kind, radius, N, H, W,
// planes): the tile shape id plus, for images with fewer tiles than the GPU
// has SMs, the number of term groups (shape | split << 8).
using TuneKey = std::tuple<int, int, int, int, int, int>;
static std::mutex g_tune_mu;
static std::map<TuneKey, int> g_tuned;
constexpr int kMaxSplit = 16;

static TuneKey tune_key(const bf_plan *p, const BfImage &img) {
    return TuneKey(p->kind, p->R, p->N, img.H, img.W, img.C);
}

// Candidate tile-shape ids of a plan (at most 4); returns their number.
static int tile_shapes(const bf_plan *p, int *ids) {
    return p->kind == BF_SPATIAL_GAUSS_TRUNC ? gauss_tile_shape_ids(p->R, ids)
                                             : box_tile_shape_ids(p->r_box, ids);
}

static cudaError_t launch_tile_config(const bf_plan *p, const BfImage &img, cudaStream_t s,
                                      int shape, int split) {
    if (p->kind == BF_SPATIAL_GAUSS_TRUNC) return launch_tile_gauss(p, img, s, shape, split);
    return launch_tile_box(p, img, s, shape, split);
}

// Output tile of a shape id (rows, columns): 0 = 32 x 64, 1 = 32 x 96,
// 2 and 3 = 64 x 64.
static void tile_dims(int shape, int *th, int *tw) {
    *th = shape >= 2 ? 64 : 32;
    *tw = shape == 1 ? 96 : 64;
}

static long long tile_count(const BfImage &img, int shape) {
    int th, tw;
    tile_dims(shape, &th, &tw);
    return (long long)((img.W + tw - 1) / tw) * ((img.H + th - 1) / th) * img.C;
}

static int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

// Whether `split` term groups suit an image of this many tiles: a power of two
// up to kMaxSplit, no more groups than terms, at most four blocks per SM in
// all, within the grid's z limit, and the 32-row tiles only (a cluster of
// the 64-row tiles' one-block-per-SM blocks would hold eight SMs).
static bool split_ok(const bf_plan *p, const BfImage &img, int shape, int split, int n_sm) {
    if (split == 1) return true;
    const long long tiles = tile_count(img, shape);
    return shape < 2 && split <= kMaxSplit && split <= (int)p->a32.size() &&
           tiles * split <= 4LL * n_sm && (long long)img.C * split <= 65535;
}

// Default term split when nothing was tuned: as many groups (a power of two)
// as bring the blocks to about two per SM.
static int default_split(const bf_plan *p, const BfImage &img, int shape) {
    const int n_sm = sm_count();
    const long long tiles = tile_count(img, shape);
    int split = 1;
    while (split * 2 <= kMaxSplit && tiles * split * 2 <= 2LL * n_sm &&
           split_ok(p, img, shape, split * 2, n_sm))
        split *= 2;
    return split;
}


// Library-owned scratch for the streaming paths (the large-radius box and the
// recursive Gaussian, forward and adjoint), one buffer per device,
// grown on demand and reused until bf_release_scratch().
static std::mutex g_scratch_mu;
static void *g_scratch[64];
static size_t g_scratch_bytes[64];

static cudaError_t get_scratch(size_t bytes, void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (g_scratch_bytes[dev] < bytes) {
        if (g_scratch[dev]) {
            e = cudaFree(g_scratch[dev]);  // synchronises with work still using it
            g_scratch[dev] = nullptr;
            g_scratch_bytes[dev] = 0;
            if (e != cudaSuccess) return e;
        }
        e = cudaMalloc(&g_scratch[dev], bytes);
        if (e != cudaSuccess) {
            g_scratch[dev] = nullptr;
            return e;
        }
        g_scratch_bytes[dev] = bytes;
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

bool tile_supported(const bf_plan *p) {
    if (p->kind == BF_SPATIAL_GAUSS_TRUNC) return gauss_tile_radius(p->R) > 0;
    return p->r_box >= 1 && p->r_box <= box_tile_max_r();
}

cudaError_t launch_tile_forward(const bf_plan *p, const BfImage &img, cudaStream_t s) {
    int cfg = -1;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(tune_key(p, img));
        if (it != g_tuned.end()) cfg = it->second;
    }
    const int shape = cfg < 0 ? 0 : (cfg & 0xff);
    const int split = cfg < 0 ? default_split(p, img, shape) : std::max(1, cfg >> 8);
    cudaError_t e = launch_tile_config(p, img, s, shape, split);
    if (split > 1 && e == cudaErrorInvalidClusterSize)
        e = launch_tile_config(p, img, s, shape, 1);  // the cluster does not fit: no split
    return e;
}

}  // namespace bf

using namespace bf;

extern "C" const char *bf_last_error(void) { return g_last_error.c_str(); }

extern "C" int bf_version(void) { return 100; }

static bf_status forward_planes(const bf_plan *plan, const BfImage &img, cudaStream_t stream,
                                const char *who);

extern "C" bf_status bf_forward(const bf_plan *plan, const void *in, bf_dtype dt, float *out,
                                int H, int W, int C, long long row_stride_elems, float *q_out,
                                cudaStream_t stream) {
    if (!plan) return fail(BF_EINVAL, "bf_forward: plan is NULL");
    if (!in || !out) return fail(BF_EINVAL, "bf_forward: in/out is NULL");
    if (H < 1 || W < 1) return fail(BF_EINVAL, "bf_forward: H and W must be >= 1");
    if (C < 1) return fail(BF_EINVAL, "bf_forward: C must be >= 1");
    if (C > 4) return fail(BF_EUNSUPPORTED, "bf_forward: at most 4 channels");
    if (dt != BF_F32 && dt != BF_U8) return fail(BF_EINVAL, "bf_forward: unknown dtype");
    if (row_stride_elems < (long long)W * C)
        return fail(BF_EINVAL, "bf_forward: row_stride_elems < W*C");
    if ((long long)H * W > (1LL << 31) / 4)
        return fail(BF_EUNSUPPORTED, "bf_forward: image too large");
    BfImage img;
    img.in = in;
    img.out = out;
    img.q_out = q_out;
    img.in_row_stride = row_stride_elems;
    img.H = H;
    img.W = W;
    img.C = C;
    img.dtype = (int)dt;
    img.q_scale = plan->q_scale;
    img.in_px = C;
    img.out_px = C;
    img.in_z = 1;
    img.out_z = 1;
    return forward_planes(plan, img, stream, "bf_forward");
}

static bf_status space_variant(const char *who, const bf_plan *plan, const void *in,
                               bf_dtype dt, const int *radius, int r_max, int hat, float *out,
                               int H, int W, int C, long long row_stride_elems,
                               cudaStream_t stream) {
    if (!plan) return fail(BF_EINVAL, std::string(who) + ": plan is NULL");
    if (!in || !out || !radius) return fail(BF_EINVAL, std::string(who) + ": a pointer is NULL");
    if (H < 1 || W < 1) return fail(BF_EINVAL, std::string(who) + ": H and W must be >= 1");
    if (C < 1 || C > 4) return fail(BF_EINVAL, std::string(who) + ": C must be 1 .. 4");
    if (hat != 0 && hat != 1) return fail(BF_EINVAL, std::string(who) + ": spatial must be 0 or 1");
    if (dt != BF_F32 && dt != BF_U8) return fail(BF_EINVAL, std::string(who) + ": unknown dtype");
    if (row_stride_elems < (long long)W * C)
        return fail(BF_EINVAL, std::string(who) + ": row_stride_elems < W * C");
    if (r_max < 0 || r_max > sv_max_radius(hat))
        return fail(BF_EINVAL, std::string(who) + ": r_max must be in [0, " +
                                   std::to_string(sv_max_radius(hat)) + "]");
    if ((long long)H * W * C > (1LL << 31) / 4)
        return fail(BF_EUNSUPPORTED, std::string(who) + ": image too large");
    if (H > BF_MAX_ROWS)
        return fail(BF_EUNSUPPORTED, std::string(who) + ": image taller than " +
                                         std::to_string(BF_MAX_ROWS) + " rows");
    return cuda_check(launch_space_variant(plan, in, (int)dt, row_stride_elems, radius, r_max,
                                           hat, out, H, W, C, stream),
                      who);
}

extern "C" bf_status bf_forward_space_variant(const bf_plan *plan, const void *in, bf_dtype dt,
                                              const int *radius, int r_max, float *out, int H,
                                              int W, long long row_stride_elems,
                                              cudaStream_t stream) {
    return space_variant("bf_forward_space_variant", plan, in, dt, radius, r_max, 0, out, H, W,
                         1, row_stride_elems, stream);
}

extern "C" bf_status bf_forward_space_variant_hat(const bf_plan *plan, const void *in,
                                                  bf_dtype dt, const int *radius, int r_max,
                                                  float *out, int H, int W,
                                                  long long row_stride_elems,
                                                  cudaStream_t stream) {
    return space_variant("bf_forward_space_variant_hat", plan, in, dt, radius, r_max, 1, out, H,
                         W, 1, row_stride_elems, stream);
}

extern "C" bf_status bf_forward_space_variant_ex(const bf_plan *plan, const void *in,
                                                 bf_dtype dt, const int *radius, int r_max,
                                                 int spatial, float *out, int H, int W, int C,
                                                 long long row_stride_elems,
                                                 cudaStream_t stream) {
    return space_variant("bf_forward_space_variant_ex", plan, in, dt, radius, r_max, spatial, out,
                         H, W, C, row_stride_elems, stream);
}

extern "C" bf_status bf_forward_host(const bf_plan *plan, const void *host_in, bf_dtype dt,
                                     void *dev_in, float *dev_out, float *host_out, int H, int W,
                                     int C, long long row_stride_elems, cudaStream_t stream) {
    if (!dev_in || !dev_out) return fail(BF_EINVAL, "bf_forward_host: dev_in/dev_out is NULL");
    if (!plan) return fail(BF_EINVAL, "bf_forward_host: plan is NULL");
    if (H < 1 || W < 1 || C < 1) return fail(BF_EINVAL, "bf_forward_host: H, W, C must be >= 1");
    if (C > 4) return fail(BF_EUNSUPPORTED, "bf_forward_host: at most 4 channels");
    if (dt != BF_F32 && dt != BF_U8) return fail(BF_EINVAL, "bf_forward_host: unknown dtype");
    if (row_stride_elems < (long long)W * C)
        return fail(BF_EINVAL, "bf_forward_host: row_stride_elems < W*C");
    if ((long long)H * W > (1LL << 31) / 4)
        return fail(BF_EUNSUPPORTED, "bf_forward_host: image too large");
    const size_t esz = dt == BF_F32 ? 4 : 1;
    const size_t in_bytes = ((size_t)(H - 1) * (size_t)row_stride_elems + (size_t)W * C) * esz;
    const size_t out_bytes = (size_t)H * W * C * sizeof(float);
    if (host_in) {
        cudaError_t e = cudaMemcpyAsync(dev_in, host_in, in_bytes, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_check(e, "bf_forward_host: host -> device copy");
    }
    const bf_status st =
        bf_forward(plan, dev_in, dt, dev_out, H, W, C, row_stride_elems, nullptr, stream);
    if (st != BF_OK) return st;
    if (host_out) {
        cudaError_t e =
            cudaMemcpyAsync(host_out, dev_out, out_bytes, cudaMemcpyDeviceToHost, stream);
        if (e != cudaSuccess) return cuda_check(e, "bf_forward_host: device -> host copy");
    }
    return BF_OK;
}

extern "C" bf_status bf_forward_host_overlap(const bf_plan *plan, const void *host_in,
                                             bf_dtype dt, void *dev_in, float *dev_out,
                                             float *host_out, int H, int W, int C,
                                             long long row_stride_elems, cudaStream_t stream,
                                             cudaStream_t copy_stream) {
    if (host_out && stream == copy_stream)
        return fail(BF_EINVAL, "bf_forward_host_overlap: copy_stream must differ from stream");
    const bf_status st = bf_forward_host(plan, host_in, dt, dev_in, dev_out, nullptr, H, W, C,
                                         row_stride_elems, stream);
    if (st != BF_OK || !host_out) return st;
    // the copy back waits for this call's filter only, on the copy stream
    cudaEvent_t done;
    cudaError_t e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_check(e, "bf_forward_host_overlap: event");
    e = cudaEventRecord(done, stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(copy_stream, done, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_out, dev_out, (size_t)H * W * C * sizeof(float),
                            cudaMemcpyDeviceToHost, copy_stream);
    cudaEventDestroy(done);  // released once the recorded work completes
    return cuda_check(e, "bf_forward_host_overlap: device -> host copy");
}

// Runs one BfImage description (interleaved channels or a stack).
static bf_status forward_planes(const bf_plan *plan, const BfImage &img, cudaStream_t stream,
                                const char *who) {
    const int H = img.H, W = img.W;
    if (H > BF_MAX_ROWS)
        return fail(BF_EUNSUPPORTED, std::string(who) + ": image taller than " +
                                         std::to_string(BF_MAX_ROWS) + " rows");
    if (tile_supported(plan))
        return cuda_check(launch_tile_forward(plan, img, stream), who);
    if (plan->kind == BF_SPATIAL_BOX_ITER) {
        void *ws = nullptr;
        cudaError_t e = get_scratch(large_workspace(plan, H, W), &ws);
        if (e == cudaErrorMemoryAllocation)
            return fail(BF_ENOMEM, std::string(who) + ": cannot allocate the large-radius scratch");
        if (e != cudaSuccess) return cuda_check(e, who);
        return cuda_check(launch_large_box(plan, img, ws, stream), who);
    }
    if (plan->kind == BF_SPATIAL_GAUSS_RECURSIVE) {
        void *ws = nullptr;
        cudaError_t e = get_scratch(recursive_workspace(plan, H, W), &ws);
        if (e == cudaErrorMemoryAllocation)
            return fail(BF_ENOMEM, std::string(who) + ": cannot allocate the recursive scratch");
        if (e != cudaSuccess) return cuda_check(e, who);
        return cuda_check(launch_recursive(plan, img, ws, stream), who);
    }
    return fail(BF_EUNSUPPORTED, std::string(who) + ": no kernel for this spatial support");
}

extern "C" bf_status bf_forward_stack(const bf_plan *plan, const void *in, bf_dtype dt,
                                      float *out, int H, int W, int count, float *q_out,
                                      cudaStream_t stream) {
    if (!plan) return fail(BF_EINVAL, "bf_forward_stack: plan is NULL");
    if (!in || !out) return fail(BF_EINVAL, "bf_forward_stack: in/out is NULL");
    if (H < 1 || W < 1 || count < 1)
        return fail(BF_EINVAL, "bf_forward_stack: H, W and count must be >= 1");
    if (dt != BF_F32 && dt != BF_U8) return fail(BF_EINVAL, "bf_forward_stack: unknown dtype");
    if ((long long)H * W > (1LL << 31) / 4 || count > 65535)
        return fail(BF_EUNSUPPORTED, "bf_forward_stack: image or stack too large");
    BfImage img;
    img.in = in;
    img.out = out;
    img.q_out = q_out;
    img.in_row_stride = W;
    img.H = H;
    img.W = W;
    img.C = count;
    img.dtype = (int)dt;
    img.q_scale = plan->q_scale;
    img.in_px = 1;
    img.out_px = 1;
    img.in_z = (long long)H * W;
    img.out_z = (long long)H * W;
    return forward_planes(plan, img, stream, "bf_forward_stack");
}

extern "C" void bf_release_scratch(void) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (int d = 0; d < 64; ++d) {
        if (g_scratch[d]) {
            cudaSetDevice(d);
            cudaFree(g_scratch[d]);
            g_scratch[d] = nullptr;
            g_scratch_bytes[d] = 0;
        }
    }
    cudaSetDevice(cur);
}

// ---- unfused baseline ---------------------------------------------------------

namespace bf {
size_t unfused_workspace(int H, int W);
cudaError_t launch_unfused(const bf_plan *pl, const float *in, float *out, int H, int W,
                           void *ws, cudaStream_t s);
}  // namespace bf

extern "C" size_t bf_forward_unfused_workspace(int H, int W) {
    if (H < 1 || W < 1) return 0;
    return unfused_workspace(H, W);
}

extern "C" bf_status bf_forward_unfused(const bf_plan *plan, const float *in, float *out, int H,
                                        int W, void *workspace, size_t workspace_bytes,
                                        cudaStream_t stream) {
    if (!plan) return fail(BF_EINVAL, "bf_forward_unfused: plan is NULL");
    if (plan->kind == BF_SPATIAL_GAUSS_RECURSIVE)
        return fail(BF_EUNSUPPORTED, "bf_forward_unfused: the unfused baseline has no "
                                     "recursive Gaussian");
    if (!in || !out || !workspace)
        return fail(BF_EINVAL, "bf_forward_unfused: in/out/workspace is NULL");
    if (H < 1 || W < 1) return fail(BF_EINVAL, "bf_forward_unfused: H and W must be >= 1");
    if ((long long)H * W > (1LL << 31) / 16)
        return fail(BF_EUNSUPPORTED, "bf_forward_unfused: image too large");
    if (workspace_bytes < unfused_workspace(H, W))
        return fail(BF_EINVAL, "bf_forward_unfused: workspace too small (need " +
                                   std::to_string(unfused_workspace(H, W)) + " bytes)");
    return cuda_check(launch_unfused(plan, in, out, H, W, workspace, stream),
                      "bf_forward_unfused launch");
}

// ---- not yet available ------------------------------------------------------

// ---- backward -------------------------------------------------------------

namespace bf {
bool bwd_supported(const bf_plan *p);
bool bwd_large_supported(const bf_plan *p);
size_t bwd_large_workspace(const bf_plan *pl, int H, int W, int count);
cudaError_t launch_backward_large(const bf_plan *pl, const float *f, const float *o,
                                  const float *q, const float *u, float *grad,
                                  double *partials, int H, int W, int count, void *ws,
                                  cudaStream_t s);
cudaError_t launch_bwd_reduce(const double *partials, int n, double *out, cudaStream_t s);
size_t bwd_blocks(int H, int W);
cudaError_t launch_backward(const bf_plan *pl, const float *f, const float *o, const float *q,
                            const float *u, float *grad, double *grad_sigma_r, double *partials,
                            int H, int W, cudaStream_t s);
cudaError_t launch_backward(const bf_plan *pl, const float *f, const float *o, const float *q,
                            const float *u, float *grad, double *grad_sigma_r, double *partials,
                            int H, int W, cudaStream_t s, int count);
}  // namespace bf

// The adjoint of either path: the fused tile kernel, or for the box with
// 8 < r <= 64 the per-term planes through the library scratch.
static bf_status run_backward(const char *who, const bf_plan *plan, const float *f,
                              const float *out, const float *q, const float *grad_out,
                              float *grad_in, double *grad_sigma_r, double *partials, int H,
                              int W, int count, cudaStream_t stream) {
    if (bwd_supported(plan))
        return cuda_check(launch_backward(plan, f, out, q, grad_out, grad_in, grad_sigma_r,
                                          partials, H, W, stream, count),
                          who);
    void *ws = nullptr;
    cudaError_t e = get_scratch(bwd_large_workspace(plan, H, W, count), &ws);
    if (e != cudaSuccess)
        return fail(BF_ENOMEM, std::string(who) + ": cannot allocate the adjoint's scratch");
    e = launch_backward_large(plan, f, out, q, grad_out, grad_in,
                              grad_sigma_r ? partials : nullptr, H, W, count, ws, stream);
    if (e == cudaSuccess && grad_sigma_r)
        e = launch_bwd_reduce(partials, (int)(bwd_blocks(H, W) * count), grad_sigma_r, stream);
    return cuda_check(e, who);
}

extern "C" size_t bf_backward_workspace(const bf_plan *plan, int H, int W) {
    if (!plan || H < 1 || W < 1) return 0;
    return bwd_blocks(H, W) * sizeof(double);
}

extern "C" size_t bf_backward_stack_workspace(const bf_plan *plan, int H, int W, int count) {
    if (!plan || H < 1 || W < 1 || count < 1) return 0;
    return bwd_blocks(H, W) * (size_t)count * sizeof(double);
}

extern "C" bf_status bf_backward_stack(const bf_plan *plan, const float *f, const float *out,
                                       const float *q, const float *grad_out, float *grad_in,
                                       double *grad_sigma_r, int H, int W, int count,
                                       void *workspace, size_t workspace_bytes,
                                       cudaStream_t stream) {
    if (!plan) return fail(BF_EINVAL, "bf_backward_stack: plan is NULL");
    if (!f || !out || !q || !grad_out || !grad_in)
        return fail(BF_EINVAL, "bf_backward_stack: a data pointer is NULL");
    if (H < 1 || W < 1 || count < 1)
        return fail(BF_EINVAL, "bf_backward_stack: H, W and count must be >= 1");
    if ((long long)H * W > (1LL << 31) / 4 || count > 65535)
        return fail(BF_EUNSUPPORTED, "bf_backward_stack: image or stack too large");
    if (H > BF_MAX_ROWS)
        return fail(BF_EUNSUPPORTED, "bf_backward_stack: image taller than " +
                                         std::to_string(BF_MAX_ROWS) + " rows");
    if (!bwd_supported(plan) && !bwd_large_supported(plan))
        return fail(BF_EUNSUPPORTED, "bf_backward_stack: no kernel for this spatial support "
                                     "(Gaussian R <= 24, box r <= 64 or the recursive "
                                     "Gaussian)");
    if (grad_sigma_r && plan->cosine)
        return fail(BF_EINVAL, "bf_backward_stack: a cosine-polynomial plan has no sigma_r; "
                               "pass grad_sigma_r = NULL");
    const size_t need = bwd_blocks(H, W) * (size_t)count * sizeof(double);
    if (grad_sigma_r) {
        if (!workspace) return fail(BF_EINVAL, "bf_backward_stack: workspace is NULL");
        if (workspace_bytes < need)
            return fail(BF_EINVAL, "bf_backward_stack: workspace too small (need " +
                                       std::to_string(need) + " bytes)");
        if ((uintptr_t)workspace % 8 != 0)
            return fail(BF_EINVAL, "bf_backward_stack: workspace must be 8-byte aligned");
    }
    return run_backward("bf_backward_stack launch", plan, f, out, q, grad_out, grad_in,
                        grad_sigma_r, reinterpret_cast<double *>(workspace), H, W, count,
                        stream);
}

extern "C" bf_status bf_backward(const bf_plan *plan, const float *f, const float *out,
                                 const float *q, const float *grad_out, float *grad_in,
                                 double *grad_sigma_r, int H, int W, void *workspace,
                                 size_t workspace_bytes, cudaStream_t stream) {
    if (!plan) return fail(BF_EINVAL, "bf_backward: plan is NULL");
    if (!f || !out || !q || !grad_out || !grad_in)
        return fail(BF_EINVAL, "bf_backward: a data pointer is NULL");
    if (H < 1 || W < 1) return fail(BF_EINVAL, "bf_backward: H and W must be >= 1");
    if ((long long)H * W > (1LL << 31) / 4)
        return fail(BF_EUNSUPPORTED, "bf_backward: image too large");
    if (H > BF_MAX_ROWS)
        return fail(BF_EUNSUPPORTED, "bf_backward: image taller than " +
                                         std::to_string(BF_MAX_ROWS) + " rows");
    if (!bwd_supported(plan) && !bwd_large_supported(plan))
        return fail(BF_EUNSUPPORTED, "bf_backward: no kernel for this spatial support "
                                     "(Gaussian R <= 24, box r <= 64 or the recursive "
                                     "Gaussian)");
    if (grad_sigma_r && plan->cosine)
        return fail(BF_EINVAL, "bf_backward: a cosine-polynomial plan has no sigma_r; "
                               "pass grad_sigma_r = NULL");
    if (grad_sigma_r) {
        if (!workspace) return fail(BF_EINVAL, "bf_backward: workspace is NULL");
        if (workspace_bytes < bwd_blocks(H, W) * sizeof(double))
            return fail(BF_EINVAL, "bf_backward: workspace too small (need " +
                                       std::to_string(bwd_blocks(H, W) * sizeof(double)) +
                                       " bytes)");
        if ((uintptr_t)workspace % 8 != 0)
            return fail(BF_EINVAL, "bf_backward: workspace must be 8-byte aligned");
    }
    return run_backward("bf_backward launch", plan, f, out, q, grad_out, grad_in,
                        grad_sigma_r, reinterpret_cast<double *>(workspace), H, W, 1, stream);
}

// ---- tile-shape autotuner ----------------------------------------------------

extern "C" bf_status bf_forward_set_shape(const bf_plan *plan, int H, int W, int C, int shape) {
    if (!plan) return fail(BF_EINVAL, "bf_forward_set_shape: NULL plan");
    if (H < 1 || W < 1 || C < 1 || C > 65535)
        return fail(BF_EINVAL, "bf_forward_set_shape: bad size (C counts the channels, or the images of a stack)");
    if (!tile_supported(plan))
        return fail(BF_EINVAL, "bf_forward_set_shape: this support runs on the streaming kernels");
    int ids[4];
    const int n = tile_shapes(plan, ids);
    bool ok = false;
    const int sid = shape & 0xff, split = std::max(1, shape >> 8);
    for (int i = 0; i < n; ++i) ok = ok || ids[i] == sid;
    if (!ok || shape < 0) return fail(BF_EINVAL, "bf_forward_set_shape: shape " +
                                                     std::to_string(sid) +
                                                     " is not available for this support");
    if ((split & (split - 1)) != 0 || split > kMaxSplit || split > (int)plan->a32.size() ||
        (long long)C * split > 65535)
        return fail(BF_EINVAL, "bf_forward_set_shape: term split " + std::to_string(split) +
                                   " must be a power of two <= 16 and <= the number of terms");
    BfImage img{};
    img.H = H;
    img.W = W;
    img.C = C;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[tune_key(plan, img)] = shape;
    return BF_OK;
}


extern "C" bf_status bf_forward_tune(const bf_plan *plan, const void *in, bf_dtype dt, float *out,
                                     int H, int W, int C, long long row_stride_elems, int reps,
                                     cudaStream_t stream, int *shape_out, float *ms_out) {
    if (!plan || !in || !out) return fail(BF_EINVAL, "bf_forward_tune: NULL argument");
    if (H < 1 || W < 1 || C < 1 || C > 4 || row_stride_elems < (long long)W * C)
        return fail(BF_EINVAL, "bf_forward_tune: bad image description");
    if (dt != BF_F32 && dt != BF_U8) return fail(BF_EINVAL, "bf_forward_tune: unknown dtype");
    if (reps < 1) reps = 3;
    BfImage img;
    img.in = in;
    img.out = out;
    img.q_out = nullptr;
    img.in_row_stride = row_stride_elems;
    img.H = H;
    img.W = W;
    img.C = C;
    img.dtype = (int)dt;
    img.q_scale = plan->q_scale;
    img.in_px = C;
    img.out_px = C;
    img.in_z = 1;
    img.out_z = 1;
    if (!tile_supported(plan)) {  // one kernel only: nothing to choose
        if (shape_out) *shape_out = -1;
        if (ms_out) *ms_out = 0.f;
        return BF_OK;
    }
    int ids[4];
    const int n = tile_shapes(plan, ids);
    const int n_sm = sm_count();
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_check(e, "bf_forward_tune");
    float best = 1e30f;
    int best_shape = 0;
    // every shape, each with every term split that suits its tile count
    for (int si = 0; si < n && e == cudaSuccess; ++si) {
        for (int split = 1; split <= kMaxSplit && e == cudaSuccess; split *= 2) {
            const int sh = ids[si];
            if (!split_ok(plan, img, sh, split, n_sm)) continue;
            e = launch_tile_config(plan, img, stream, sh, split);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
            for (int k = 0; k < reps && e == cudaSuccess; ++k)
                e = launch_tile_config(plan, img, stream, sh, split);
            if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            if (e == cudaSuccess && ms < best) {
                best = ms;
                best_shape = sh | (split > 1 ? split << 8 : 0);
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_check(e, "bf_forward_tune");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[tune_key(plan, img)] = best_shape;
    }
    if (shape_out) *shape_out = best_shape;
    if (ms_out) *ms_out = best;
    return BF_OK;
}

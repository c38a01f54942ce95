// Batched forward: many single-channel f32 images of uneven sizes, each with
// its own plan, replayed from one CUDA graph.
//
// Images whose box half-width r fits a tile (r <= 8): the host flattens them
// into tiles, orders the tiles largest cost first (longest-processing-time
// order: cost ~ terms x tile area including the halo), and uploads the queue
// with a per-image descriptor and term table.  Each resident block of the
// persistent kernel claims the next tile with one atomicAdd and runs the
// fused tile body of that image's r (one instantiation per r), so small and
// large images, cheap and expensive plans share the GPU without a tail of
// idle SMs per image.  The claim loop is bounded by the number of tiles; a
// block that would exceed it sets the device error flag instead.
//
// Images with 8 < r <= 64: the streaming sweeps of the single-image path,
// spread over kBatchLanes chains (largest cost first onto the least loaded);
// the images of a chain run one after the other through that chain's
// scratch, the chains and the persistent launch run concurrently.
//
// The counter reset, the persistent launch and the chains are captured into
// a CUDA graph (again after every bind, which changes the streaming images'
// pointers) and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "bf_tile.cuh"

namespace bf {

namespace {

constexpr int kBatchNT = 256;
constexpr int kBatchTileMaxR = 8;  // larger half-widths take the streaming sweeps
constexpr int kBatchMaxR = 64;
constexpr int kBatchLanes = 4;     // concurrent chains of streaming images

// tile shape of the batch bodies; every body uses kBatchNT threads
template <int R>
struct BatchShape {
    static constexpr int TH = 32;
    static constexpr int TW = 64;
    static constexpr int TWT = 16;
    using G = TileGeom<1, R, TH, TW, TWT>;
    static_assert(G::NT == kBatchNT, "batch bodies share one block size");
};

constexpr int kBatchTH = 32;
constexpr int kBatchTW = 64;

struct ImgDesc {
    const float *in;
    float *out;
    int H, W, r, n_terms, term_off, tiles_x;
    float q_scale;
};

struct BatchParams {
    const ImgDesc *imgs;
    const int4 *queue;  // (image, tile x, tile y, 0)
    int n_tiles;
    int *counter;
    int *err;
    const float *ta;    // term weights, all images
    const float *tt;    // term frequencies (turns per gray level)
};

template <int R>
__device__ __forceinline__ void run_tile(const BatchParams &p, const ImgDesc &d, int tx, int ty,
                                         float *smem) {
    using S = BatchShape<R>;
    TileJob jb;
    jb.in = d.in;
    jb.out = d.out;
    jb.q_out = nullptr;
    jb.in_row_stride = d.W;
    jb.H = d.H;
    jb.W = d.W;
    jb.in_px = 1;
    jb.out_px = 1;
    jb.dtype = 0;
    jb.q_scale = d.q_scale;
    jb.a = p.ta + d.term_off;
    jb.t = p.tt + d.term_off;
    jb.n_terms = d.n_terms;
    jb.w2 = nullptr;
    jb.x0 = tx * S::TW;
    jb.y0 = ty * S::TH;
    jb.split = 1;
    tile_body<1, R, S::TH, S::TW, S::TWT>(jb, smem);
}

template <int... Rs>
struct MaxSmem;
template <int R>
struct MaxSmem<R> {
    static constexpr size_t v = BatchShape<R>::G::SMEM;
};
template <int R, int... Rs>
struct MaxSmem<R, Rs...> {
    static constexpr size_t v =
        BatchShape<R>::G::SMEM > MaxSmem<Rs...>::v ? BatchShape<R>::G::SMEM : MaxSmem<Rs...>::v;
};
constexpr size_t kBatchSmem = MaxSmem<1, 2, 3, 4, 5, 6, 7, 8>::v;
static_assert(kBatchSmem <= 227 * 1024, "batch shared memory");

__global__ void __launch_bounds__(kBatchNT, 2) bf_batch_persist(const __grid_constant__ BatchParams p) {
    extern __shared__ float4 sm4[];
    float *smem = reinterpret_cast<float *>(sm4);
    __shared__ int s_tile;
    for (int it = 0; it <= p.n_tiles; ++it) {
        __syncthreads();  // the previous tile and s_tile are no longer in use
        if (threadIdx.x == 0) s_tile = atomicAdd(p.counter, 1);
        __syncthreads();
        const int t = s_tile;
        if (t >= p.n_tiles) return;
        if (it == p.n_tiles) {  // more claims than tiles: cannot happen unless the queue is corrupt
            if (threadIdx.x == 0) atomicExch(p.err, 1);
            return;
        }
        const int4 w = p.queue[t];
        const ImgDesc d = p.imgs[w.x];
        switch (d.r) {
            case 1: run_tile<1>(p, d, w.y, w.z, smem); break;
            case 2: run_tile<2>(p, d, w.y, w.z, smem); break;
            case 3: run_tile<3>(p, d, w.y, w.z, smem); break;
            case 4: run_tile<4>(p, d, w.y, w.z, smem); break;
            case 5: run_tile<5>(p, d, w.y, w.z, smem); break;
            case 6: run_tile<6>(p, d, w.y, w.z, smem); break;
            case 7: run_tile<7>(p, d, w.y, w.z, smem); break;
            case 8: run_tile<8>(p, d, w.y, w.z, smem); break;
            default:
                if (threadIdx.x == 0) atomicExch(p.err, 2);
                break;
        }
    }
}

}  // namespace

}  // namespace bf

using namespace bf;

struct bf_batch {
    int count = 0;
    int dev = 0;
    std::vector<ImgDesc> h_imgs;
    std::vector<int4> h_queue_lpt, h_queue_rowmajor;
    ImgDesc *d_imgs = nullptr;
    int4 *d_queue = nullptr;
    int *d_counter = nullptr;
    int *d_err = nullptr;
    float *d_ta = nullptr, *d_tt = nullptr;
    int n_tiles = 0;
    int grid = 0;
    int order = 0;  // 0: largest cost first, 1: image by image
    bool bound = false;
    // images with r > kBatchTileMaxR: their index, a copy of their plan, the
    // chain (lane) each runs in, and one scratch per lane (the images of a
    // lane run one after the other)
    std::vector<int> stream_ids;
    std::vector<bf_plan> stream_plans;
    std::vector<int> stream_lane;
    int n_lanes = 0;
    void *d_scratch[kBatchLanes] = {};
    cudaStream_t cap = nullptr;  // private stream the graph is captured on
    cudaStream_t lane_stream[kBatchLanes] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kBatchLanes] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void batch_free(bf_batch *b) {
    if (!b) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(b->dev);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_imgs);
    cudaFree(b->d_queue);
    cudaFree(b->d_counter);
    cudaFree(b->d_err);
    cudaFree(b->d_ta);
    cudaFree(b->d_tt);
    for (int k = 0; k < kBatchLanes; ++k) {
        cudaFree(b->d_scratch[k]);
        if (b->lane_stream[k]) cudaStreamDestroy(b->lane_stream[k]);
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaSetDevice(cur);
    delete b;
}

// (Re)build the graph by capturing, on the batch's private stream: the
// counter reset and the persistent kernel (if any image is tiled), then the
// streaming sweeps of every image with r > kBatchTileMaxR once the batch is
// bound (before that their pointers are unknown).
static cudaError_t batch_build_graph(bf_batch *b) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaError_t e = cudaSuccess;
    if (!b->cap) {
        e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
        for (int k = 0; k < b->n_lanes && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithFlags(&b->lane_stream[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return e;
    }
    const bool streaming = b->bound && !b->stream_ids.empty();
    if (b->n_tiles == 0 && !streaming) return cudaSuccess;  // nothing to replay yet
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    if (streaming) {
        // fork the lanes off the capture stream
        le = cudaEventRecord(b->ev_fork, b->cap);
        for (int k = 0; k < b->n_lanes && le == cudaSuccess; ++k)
            le = cudaStreamWaitEvent(b->lane_stream[k], b->ev_fork, 0);
    }
    if (b->n_tiles > 0 && le == cudaSuccess) {
        le = cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->cap);
        BatchParams prm;
        prm.imgs = b->d_imgs;
        prm.queue = b->d_queue;
        prm.n_tiles = b->n_tiles;
        prm.counter = b->d_counter;
        prm.err = b->d_err;
        prm.ta = b->d_ta;
        prm.tt = b->d_tt;
        if (le == cudaSuccess) {
            bf_batch_persist<<<b->grid, kBatchNT, kBatchSmem, b->cap>>>(prm);
            le = cudaGetLastError();
        }
    }
    if (streaming) {
        for (size_t k = 0; k < b->stream_ids.size() && le == cudaSuccess; ++k) {
            const ImgDesc &d = b->h_imgs[b->stream_ids[k]];
            BfImage img;
            img.in = d.in;
            img.out = d.out;
            img.q_out = nullptr;
            img.in_row_stride = d.W;
            img.H = d.H;
            img.W = d.W;
            img.C = 1;
            img.dtype = 0;
            img.q_scale = d.q_scale;
            img.in_px = 1;
            img.out_px = 1;
            img.in_z = 1;
            img.out_z = 1;
            const int lane = b->stream_lane[k];
            le = launch_large_box(&b->stream_plans[k], img, b->d_scratch[lane],
                                  b->lane_stream[lane]);
        }
        // join every lane back
        for (int k = 0; k < b->n_lanes && le == cudaSuccess; ++k) {
            le = cudaEventRecord(b->ev_join[k], b->lane_stream[k]);
            if (le == cudaSuccess) le = cudaStreamWaitEvent(b->cap, b->ev_join[k], 0);
        }
    }
    e = cudaStreamEndCapture(b->cap, &b->graph);
    if (le != cudaSuccess) return le;
    if (e != cudaSuccess) return e;
    return cudaGraphInstantiate(&b->exec, b->graph, 0);
}

static cudaError_t batch_upload_queue(bf_batch *b, cudaStream_t s) {
    const std::vector<int4> &q = b->order == 0 ? b->h_queue_lpt : b->h_queue_rowmajor;
    return cudaMemcpyAsync(b->d_queue, q.data(), sizeof(int4) * q.size(), cudaMemcpyHostToDevice, s);
}

extern "C" bf_status bf_batch_create(bf_batch **out, const bf_plan *const *plans, const int *H,
                                     const int *W, int count) {
    if (!out) return fail(BF_EINVAL, "bf_batch_create: out is NULL");
    *out = nullptr;
    if (!plans || !H || !W || count < 1)
        return fail(BF_EINVAL, "bf_batch_create: plans/H/W NULL or count < 1");
    for (int i = 0; i < count; ++i) {
        if (!plans[i]) return fail(BF_EINVAL, "bf_batch_create: a plan is NULL");
        if (H[i] < 1 || W[i] < 1) return fail(BF_EINVAL, "bf_batch_create: a size is < 1");
        if ((long long)H[i] * W[i] > (1LL << 31) / 4)
            return fail(BF_EUNSUPPORTED, "bf_batch_create: an image is too large");
        if (plans[i]->kind != BF_SPATIAL_BOX_ITER || plans[i]->r_box < 1 ||
            plans[i]->r_box > kBatchMaxR)
            return fail(BF_EUNSUPPORTED,
                        "bf_batch_create: the batch serves the 3-pass box with 1 <= r <= 64");
    }
    bf_batch *b = new (std::nothrow) bf_batch();
    if (!b) return fail(BF_ENOMEM, "bf_batch_create: out of host memory");
    cudaError_t e = cudaGetDevice(&b->dev);
    if (e != cudaSuccess) {
        delete b;
        return cuda_check(e, "bf_batch_create");
    }
    b->count = count;
    std::vector<float> ta, tt;
    struct Cost {
        double c;
        int4 w;
    };
    std::vector<Cost> tiles;
    std::vector<size_t> stream_ws;  // scratch each streaming image needs
    for (int i = 0; i < count; ++i) {
        const bf_plan *pl = plans[i];
        ImgDesc d{};
        d.H = H[i];
        d.W = W[i];
        d.r = pl->r_box;
        d.n_terms = (int)pl->a32.size();
        d.term_off = (int)ta.size();
        d.q_scale = pl->q_scale;
        if (d.r > kBatchTileMaxR) {
            b->h_imgs.push_back(d);
            b->stream_ids.push_back(i);
            b->stream_plans.push_back(*pl);
            stream_ws.push_back(large_workspace(pl, H[i], W[i]));
            continue;
        }
        const int th = kBatchTH;
        d.tiles_x = (W[i] + kBatchTW - 1) / kBatchTW;
        const int tiles_y = (H[i] + th - 1) / th;
        for (int k = 0; k < d.n_terms; ++k) {
            ta.push_back(pl->a32[k]);
            tt.push_back(pl->turns32[k]);
        }
        b->h_imgs.push_back(d);
        const double cost = (double)d.n_terms * (th + 6.0 * d.r) * (kBatchTW + 6.0 * d.r);
        for (int ty = 0; ty < tiles_y; ++ty)
            for (int tx = 0; tx < d.tiles_x; ++tx) {
                const int4 w = make_int4(i, tx, ty, 0);
                tiles.push_back({cost, w});
                b->h_queue_rowmajor.push_back(w);
            }
    }
    std::stable_sort(tiles.begin(), tiles.end(),
                     [](const Cost &x, const Cost &y) { return x.c > y.c; });
    // streaming images onto lanes, largest cost first onto the least loaded
    {
        const int ns = (int)b->stream_ids.size();
        b->n_lanes = std::min(kBatchLanes, ns);
        b->stream_lane.assign(ns, 0);
        std::vector<int> order(ns);
        for (int k = 0; k < ns; ++k) order[k] = k;
        auto cost = [&](int k) {
            const ImgDesc &d = b->h_imgs[b->stream_ids[k]];
            return (double)d.n_terms * d.H * d.W;
        };
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
        std::vector<double> load(std::max(1, b->n_lanes), 0.0);
        for (int k : order) {
            const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            b->stream_lane[k] = l;
            load[l] += cost(k);
        }
    }
    size_t lane_ws[kBatchLanes] = {};
    for (size_t k = 0; k < b->stream_ids.size(); ++k)
        lane_ws[b->stream_lane[k]] = std::max(lane_ws[b->stream_lane[k]], stream_ws[k]);
    for (auto &c : tiles) b->h_queue_lpt.push_back(c.w);
    b->n_tiles = (int)tiles.size();

    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(bf_batch_persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kBatchSmem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bf_batch_persist, kBatchNT,
                                                          kBatchSmem);
    if (e == cudaSuccess) {
        b->grid = std::max(1, std::min(sms * std::max(per_sm, 1), b->n_tiles));
        size_t nq = sizeof(int4) * (size_t)std::max(1, b->n_tiles);
        e = cudaMalloc(&b->d_imgs, sizeof(ImgDesc) * count);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, nq);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_ta, sizeof(float) * std::max<size_t>(1, ta.size()));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_tt, sizeof(float) * std::max<size_t>(1, tt.size()));
        for (int k = 0; k < b->n_lanes && e == cudaSuccess; ++k)
            e = cudaMalloc(&b->d_scratch[k], lane_ws[k]);
    }
    if (e == cudaSuccess && b->n_tiles > 0)
        e = cudaMemcpy(b->d_queue, b->h_queue_lpt.data(), sizeof(int4) * b->n_tiles,
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !ta.empty())
        e = cudaMemcpy(b->d_ta, ta.data(), sizeof(float) * ta.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !tt.empty())
        e = cudaMemcpy(b->d_tt, tt.data(), sizeof(float) * tt.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = batch_build_graph(b);
    if (e != cudaSuccess) {
        batch_free(b);
        if (e == cudaErrorMemoryAllocation)
            return fail(BF_ENOMEM, "bf_batch_create: device allocation failed");
        return cuda_check(e, "bf_batch_create");
    }
    *out = b;
    return BF_OK;
}

extern "C" bf_status bf_batch_bind(bf_batch *b, const float *const *in, float *const *out,
                                   cudaStream_t stream) {
    if (!b) return fail(BF_EINVAL, "bf_batch_bind: batch is NULL");
    if (!in || !out) return fail(BF_EINVAL, "bf_batch_bind: in/out is NULL");
    for (int i = 0; i < b->count; ++i) {
        if (!in[i] || !out[i]) return fail(BF_EINVAL, "bf_batch_bind: an image pointer is NULL");
        b->h_imgs[i].in = in[i];
        b->h_imgs[i].out = out[i];
    }
    cudaError_t e = cudaMemcpyAsync(b->d_imgs, b->h_imgs.data(), sizeof(ImgDesc) * b->count,
                                    cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // h_imgs may change on the next bind
    if (e != cudaSuccess) return cuda_check(e, "bf_batch_bind");
    const bool was_bound = b->bound;
    b->bound = true;
    if (!b->stream_ids.empty() || !was_bound) {
        // the streaming images' pointers live in the graph: capture it again
        e = batch_build_graph(b);
        if (e != cudaSuccess) {
            b->bound = false;
            return cuda_check(e, "bf_batch_bind");
        }
    }
    return BF_OK;
}

extern "C" bf_status bf_batch_forward(bf_batch *b, cudaStream_t stream) {
    if (!b) return fail(BF_EINVAL, "bf_batch_forward: batch is NULL");
    if (!b->bound || !b->exec) return fail(BF_EINVAL, "bf_batch_forward: call bf_batch_bind first");
    return cuda_check(cudaGraphLaunch(b->exec, stream), "bf_batch_forward");
}

extern "C" bf_status bf_batch_check(bf_batch *b, cudaStream_t stream, int *device_error) {
    if (!b || !device_error) return fail(BF_EINVAL, "bf_batch_check: NULL argument");
    cudaError_t e = cudaStreamSynchronize(stream);
    int v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, b->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_check(e, "bf_batch_check");
    *device_error = v;
    return BF_OK;
}

extern "C" void bf_batch_destroy(bf_batch *b) { batch_free(b); }

// Launch-configuration autotuner for a bound batch: times the graph for each
// candidate (persistent grid of 1x or 2x the resident blocks, queue in
// largest-cost-first or image order), keeps the fastest, and reports it.
extern "C" bf_status bf_batch_tune(bf_batch *b, cudaStream_t stream, int reps, int *grid_out,
                                   int *order_out, float *ms_out) {
    if (!b) return fail(BF_EINVAL, "bf_batch_tune: batch is NULL");
    if (!b->bound) return fail(BF_EINVAL, "bf_batch_tune: call bf_batch_bind first");
    if (reps < 1) reps = 3;
    int sms = 0, per_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bf_batch_persist, kBatchNT,
                                                          kBatchSmem);
    if (e != cudaSuccess) return cuda_check(e, "bf_batch_tune");
    const int resident = sms * std::max(per_sm, 1);
    const int grids[2] = {std::min(resident, b->n_tiles), std::min(2 * resident, b->n_tiles)};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_grid = b->grid, best_order = b->order;
    for (int order = 0; order < 2 && e == cudaSuccess; ++order) {
        for (int gi = 0; gi < 2 && e == cudaSuccess; ++gi) {
            b->order = order;
            b->grid = std::max(1, grids[gi]);
            e = batch_upload_queue(b, stream);
            if (e == cudaSuccess) e = batch_build_graph(b);
            if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, stream);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
            for (int k = 0; k < reps && e == cudaSuccess; ++k) e = cudaGraphLaunch(b->exec, stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            if (e == cudaSuccess && ms < best) {
                best = ms;
                best_grid = b->grid;
                best_order = order;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_check(e, "bf_batch_tune");
    b->order = best_order;
    b->grid = best_grid;
    e = batch_upload_queue(b, stream);
    if (e == cudaSuccess) e = batch_build_graph(b);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_check(e, "bf_batch_tune");
    if (grid_out) *grid_out = best_grid;
    if (order_out) *order_out = best_order;
    if (ms_out) *ms_out = best;
    return BF_OK;
}

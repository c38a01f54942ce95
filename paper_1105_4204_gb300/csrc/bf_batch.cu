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
// Images with 8 < r <= 64, and the recursive Gaussian's: the streaming sweeps
// of the single-image path,
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
constexpr int kBatchMaxSplit = 4;  // most term groups of a batch tile

// Tile shapes of the batch bodies (ids as bf_forward's), all of kBatchNT
// threads: 0 = 32 x 64 tiles, 16-pixel row segments (8 pixels per thread);
// 1 = 32 x 96, 24-pixel segments (12 pixels per thread, r <= 4); 3 = 64 x 64,
// 32-pixel segments (16 pixels per thread, r = 7, 8).
template <int R, int SH>
struct BatchShape {
    static constexpr int TH = SH == 3 ? 64 : 32;
    static constexpr int TW = SH == 1 ? 96 : 64;
    static constexpr int TWT = SH == 1 ? 24 : (SH == 3 ? 32 : 16);
    using G = TileGeom<1, R, TH, TW, TWT>;
    static_assert(G::NT == kBatchNT, "batch bodies share one block size");
};

__host__ __device__ constexpr bool batch_shape_ok(int r, int sh) {
    return sh == 0 || (sh == 1 && r <= 4) || (sh == 3 && r >= 7 && r <= 8);
}

struct ImgDesc {
    const float *in;
    float *out;
    int H, W, r, n_terms, term_off, tiles_x;
    int shape, split;  // the configuration of its radius bucket
    float q_scale;
    float *slots;      // split > 1: 2 * split planes of H * W (P, Q per group)
};

struct BatchParams {
    const ImgDesc *imgs;
    const int4 *queue;  // (image, tile x, tile y, term group)
    int n_tiles;
    int *counter;
    int *err;
    const float *ta;    // term weights, all images
    const float *tt;    // term frequencies (turns per gray level)
};

template <int R, int SH>
__device__ __forceinline__ void run_tile(const BatchParams &p, const ImgDesc &d, const int4 &w,
                                         float *smem) {
    using S = BatchShape<R, SH>;
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
    // term group w.w of d.split (the cut bf_forward's term split makes)
    const int m0 = w.w * d.n_terms / d.split, m1 = (w.w + 1) * d.n_terms / d.split;
    jb.a = p.ta + d.term_off + m0;
    jb.t = p.tt + d.term_off + m0;
    jb.n_terms = m1 - m0;
    jb.w2 = nullptr;
    jb.x0 = w.y * S::TW;
    jb.y0 = w.z * S::TH;
    jb.split = 1;
    const long long n = (long long)d.H * d.W;
    jb.slot = d.split > 1 ? d.slots + 2LL * w.w * n : nullptr;
    jb.slot_n = n;
    tile_body<1, R, S::TH, S::TW, S::TWT>(jb, smem);
}

// Shared memory of the tile body of half-width r and shape sh.
size_t batch_body_smem(int r, int sh) {
    switch (r * 4 + sh) {
        case 1 * 4 + 0: return BatchShape<1, 0>::G::SMEM;
        case 2 * 4 + 0: return BatchShape<2, 0>::G::SMEM;
        case 3 * 4 + 0: return BatchShape<3, 0>::G::SMEM;
        case 4 * 4 + 0: return BatchShape<4, 0>::G::SMEM;
        case 5 * 4 + 0: return BatchShape<5, 0>::G::SMEM;
        case 6 * 4 + 0: return BatchShape<6, 0>::G::SMEM;
        case 7 * 4 + 0: return BatchShape<7, 0>::G::SMEM;
        case 8 * 4 + 0: return BatchShape<8, 0>::G::SMEM;
        case 1 * 4 + 1: return BatchShape<1, 1>::G::SMEM;
        case 2 * 4 + 1: return BatchShape<2, 1>::G::SMEM;
        case 3 * 4 + 1: return BatchShape<3, 1>::G::SMEM;
        case 4 * 4 + 1: return BatchShape<4, 1>::G::SMEM;
        case 7 * 4 + 3: return BatchShape<7, 3>::G::SMEM;
        case 8 * 4 + 3: return BatchShape<8, 3>::G::SMEM;
        default: return 0;
    }
}

// Persistent kernel.  WIDE: the variant with the 64 x 64 bodies (one block
// per SM, all registers); otherwise two blocks per SM and 128 registers.
template <bool WIDE>
__global__ void __launch_bounds__(kBatchNT, WIDE ? 1 : 2)
    bf_batch_persist(const __grid_constant__ BatchParams p) {
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
        const int key = d.r * 4 + d.shape;  // uniform over the block
        switch (key) {
            case 1 * 4 + 0: run_tile<1, 0>(p, d, w, smem); break;
            case 2 * 4 + 0: run_tile<2, 0>(p, d, w, smem); break;
            case 3 * 4 + 0: run_tile<3, 0>(p, d, w, smem); break;
            case 4 * 4 + 0: run_tile<4, 0>(p, d, w, smem); break;
            case 5 * 4 + 0: run_tile<5, 0>(p, d, w, smem); break;
            case 6 * 4 + 0: run_tile<6, 0>(p, d, w, smem); break;
            case 7 * 4 + 0: run_tile<7, 0>(p, d, w, smem); break;
            case 8 * 4 + 0: run_tile<8, 0>(p, d, w, smem); break;
            case 1 * 4 + 1: run_tile<1, 1>(p, d, w, smem); break;
            case 2 * 4 + 1: run_tile<2, 1>(p, d, w, smem); break;
            case 3 * 4 + 1: run_tile<3, 1>(p, d, w, smem); break;
            case 4 * 4 + 1: run_tile<4, 1>(p, d, w, smem); break;
            case 7 * 4 + 3:
                if constexpr (WIDE) run_tile<7, 3>(p, d, w, smem);
                else if (threadIdx.x == 0) atomicExch(p.err, 2);
                break;
            case 8 * 4 + 3:
                if constexpr (WIDE) run_tile<8, 3>(p, d, w, smem);
                else if (threadIdx.x == 0) atomicExch(p.err, 2);
                break;
            default:
                if (threadIdx.x == 0) atomicExch(p.err, 2);
                break;
        }
    }
}

// Term-split images: out = sum of the groups' P / sum of their Q, groups in
// order.  blockIdx.y: the image's index in the list.
struct SplitDesc {
    const float *slots;
    float *out;
    long long n;
    int split;
};

__global__ void batch_split_final(const SplitDesc *__restrict__ list) {
    const SplitDesc d = list[blockIdx.y];
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d.n; i += step) {
        float pv = d.slots[i], qv = d.slots[d.n + i];
        for (int g = 1; g < d.split; ++g) {
            pv += d.slots[2 * g * d.n + i];
            qv += d.slots[(2 * g + 1) * d.n + i];
        }
        d.out[i] = pv / qv;
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
    size_t queue_cap = 0;  // int4 entries d_queue holds
    int *d_counter = nullptr;
    int *d_err = nullptr;
    float *d_ta = nullptr, *d_tt = nullptr;
    int n_tiles = 0;
    int grid = 0;
    int order = 0;  // 0: largest cost first, 1: image by image
    bool bound = false;
    // configuration of each tile radius bucket r = 1 .. kBatchTileMaxR:
    // tile shape id and number of term groups per tile
    int cfg_shape[kBatchTileMaxR + 1] = {};
    int cfg_split[kBatchTileMaxR + 1] = {};
    bool wide = false;   // a bucket uses the 64 x 64 bodies: the one-block-per-SM kernel
    size_t smem = 0;     // dynamic shared memory of the persistent launch
    int resident = 0;    // resident blocks of that launch
    // term-split images: partial sums and the list the final kernel reads
    float *d_slots = nullptr;
    size_t slots_cap = 0;  // floats
    SplitDesc *d_split = nullptr;
    int n_split = 0;
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
    cudaFree(b->d_slots);
    cudaFree(b->d_split);
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

static void tile_dims_batch(int shape, int *th, int *tw) {
    *th = shape == 3 ? 64 : 32;
    *tw = shape == 1 ? 96 : 64;
}

// Applies the buckets' configuration to the tiled images: their shape, split,
// tile counts and slot planes; the tile queue in largest-cost-first and in
// image order (cost ~ terms of the work item x tile area with its halo); the
// persistent kernel variant, its shared memory and resident blocks; and the
// list of term-split images for the final kernel (whose outputs are known
// once bound).  Uploads the image table and the queue (synchronously).
static cudaError_t batch_apply_config(bf_batch *b) {
    struct Cost {
        double c;
        int4 w;
    };
    std::vector<Cost> items;
    b->h_queue_rowmajor.clear();
    b->h_queue_lpt.clear();
    b->wide = false;
    b->smem = 0;
    size_t slot_floats = 0;
    for (int i = 0; i < b->count; ++i) {
        ImgDesc &d = b->h_imgs[i];
        if (d.r > kBatchTileMaxR) continue;
        d.shape = b->cfg_shape[d.r];
        d.split = std::max(1, std::min(b->cfg_split[d.r], d.n_terms));
        if (d.shape == 3) b->wide = true;
        b->smem = std::max(b->smem, batch_body_smem(d.r, d.shape));
        int th, tw;
        tile_dims_batch(d.shape, &th, &tw);
        d.tiles_x = (d.W + tw - 1) / tw;
        const int tiles_y = (d.H + th - 1) / th;
        if (d.split > 1) slot_floats += 2 * (size_t)d.split * d.H * d.W;
        for (int g = 0; g < d.split; ++g) {
            const int nt = (g + 1) * d.n_terms / d.split - g * d.n_terms / d.split;
            const double cost = (double)nt * (th + 6.0 * d.r) * (tw + 6.0 * d.r);
            for (int ty = 0; ty < tiles_y; ++ty)
                for (int tx = 0; tx < d.tiles_x; ++tx) {
                    const int4 w = make_int4(i, tx, ty, g);
                    items.push_back({cost, w});
                    b->h_queue_rowmajor.push_back(w);
                }
        }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const Cost &x, const Cost &y) { return x.c > y.c; });
    for (auto &c : items) b->h_queue_lpt.push_back(c.w);
    b->n_tiles = (int)items.size();
    cudaError_t e = cudaSuccess;
    if ((size_t)b->n_tiles > b->queue_cap) {
        cudaFree(b->d_queue);
        b->d_queue = nullptr;
        b->queue_cap = 0;
        e = cudaMalloc(&b->d_queue, sizeof(int4) * (size_t)b->n_tiles);
        if (e != cudaSuccess) return e;
        b->queue_cap = b->n_tiles;
    }
    if (slot_floats > b->slots_cap) {
        cudaFree(b->d_slots);
        b->d_slots = nullptr;
        b->slots_cap = 0;
        e = cudaMalloc(&b->d_slots, sizeof(float) * slot_floats);
        if (e != cudaSuccess) return e;
        b->slots_cap = slot_floats;
    }
    // slot planes and the final kernel's list
    std::vector<SplitDesc> list;
    size_t off = 0;
    for (int i = 0; i < b->count; ++i) {
        ImgDesc &d = b->h_imgs[i];
        d.slots = nullptr;
        if (d.r > kBatchTileMaxR || d.split <= 1) continue;
        d.slots = b->d_slots + off;
        off += 2 * (size_t)d.split * d.H * d.W;
        list.push_back({d.slots, d.out, (long long)d.H * d.W, d.split});
    }
    b->n_split = (int)list.size();
    cudaFree(b->d_split);
    b->d_split = nullptr;
    if (!list.empty()) {
        e = cudaMalloc(&b->d_split, sizeof(SplitDesc) * list.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_split, list.data(), sizeof(SplitDesc) * list.size(),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    auto kern = b->wide ? bf_batch_persist<true> : bf_batch_persist<false>;
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchNT, b->smem);
    if (e != cudaSuccess) return e;
    b->resident = sms * std::max(per_sm, 1);
    b->grid = std::max(1, std::min(b->resident, b->n_tiles));
    e = cudaMemcpy(b->d_imgs, b->h_imgs.data(), sizeof(ImgDesc) * b->count,
                   cudaMemcpyHostToDevice);
    if (e == cudaSuccess && b->n_tiles > 0) {
        const std::vector<int4> &q = b->order == 0 ? b->h_queue_lpt : b->h_queue_rowmajor;
        e = cudaMemcpy(b->d_queue, q.data(), sizeof(int4) * q.size(), cudaMemcpyHostToDevice);
    }
    return e;
}

// (Re)build the graph by capturing, on the batch's private stream: the
// counter reset, the persistent kernel and the final sum of the term-split
// images (if any image is tiled), then the streaming sweeps of every image
// with r > kBatchTileMaxR once the batch is bound (before that their pointers
// are unknown).
// The tiled images' work on `stream`: the claim counter reset, the persistent
// launch and, for term-split images, the sum over the groups.
static cudaError_t batch_launch_tiles(bf_batch *b, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
    BatchParams prm;
    prm.imgs = b->d_imgs;
    prm.queue = b->d_queue;
    prm.n_tiles = b->n_tiles;
    prm.counter = b->d_counter;
    prm.err = b->d_err;
    prm.ta = b->d_ta;
    prm.tt = b->d_tt;
    if (b->wide)
        bf_batch_persist<true><<<b->grid, kBatchNT, b->smem, stream>>>(prm);
    else
        bf_batch_persist<false><<<b->grid, kBatchNT, b->smem, stream>>>(prm);
    e = cudaGetLastError();
    if (e == cudaSuccess && b->n_split > 0) {
        batch_split_final<<<dim3(64, b->n_split), 256, 0, stream>>>(b->d_split);
        e = cudaGetLastError();
    }
    return e;
}

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
    if (b->n_tiles > 0 && le == cudaSuccess) le = batch_launch_tiles(b, b->cap);
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
            const bf_plan *sp = &b->stream_plans[k];
            le = sp->kind == BF_SPATIAL_GAUSS_RECURSIVE
                     ? launch_recursive(sp, img, b->d_scratch[lane], b->lane_stream[lane])
                     : launch_large_box(sp, img, b->d_scratch[lane], b->lane_stream[lane]);
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
        const bool box_ok = plans[i]->kind == BF_SPATIAL_BOX_ITER && plans[i]->r_box >= 1 &&
                            plans[i]->r_box <= kBatchMaxR;
        if (!box_ok && plans[i]->kind != BF_SPATIAL_GAUSS_RECURSIVE)
            return fail(BF_EUNSUPPORTED,
                        "bf_batch_create: the batch serves the 3-pass box with 1 <= r <= 64 "
                        "and the recursive Gaussian");
    }
    bf_batch *b = new (std::nothrow) bf_batch();
    if (!b) return fail(BF_ENOMEM, "bf_batch_create: out of host memory");
    cudaError_t e = cudaGetDevice(&b->dev);
    if (e != cudaSuccess) {
        delete b;
        return cuda_check(e, "bf_batch_create");
    }
    b->count = count;
    for (int r = 0; r <= kBatchTileMaxR; ++r) {
        b->cfg_shape[r] = 0;
        b->cfg_split[r] = 1;
    }
    std::vector<float> ta, tt;
    std::vector<size_t> stream_ws;  // scratch each streaming image needs
    for (int i = 0; i < count; ++i) {
        const bf_plan *pl = plans[i];
        ImgDesc d{};
        d.H = H[i];
        d.W = W[i];
        // the streaming images (box r > 8, and the recursive Gaussian, which
        // carries r = kBatchTileMaxR + 1) run on the lanes, not in the tile queue
        const bool rec = pl->kind == BF_SPATIAL_GAUSS_RECURSIVE;
        d.r = rec ? kBatchTileMaxR + 1 : pl->r_box;
        d.n_terms = (int)pl->a32.size();
        d.term_off = (int)ta.size();
        d.q_scale = pl->q_scale;
        d.split = 1;
        if (d.r > kBatchTileMaxR) {
            b->h_imgs.push_back(d);
            b->stream_ids.push_back(i);
            b->stream_plans.push_back(*pl);
            stream_ws.push_back(rec ? recursive_workspace(pl, H[i], W[i])
                                    : large_workspace(pl, H[i], W[i]));
            continue;
        }
        for (int k = 0; k < d.n_terms; ++k) {
            ta.push_back(pl->a32[k]);
            tt.push_back(pl->turns32[k]);
        }
        b->h_imgs.push_back(d);
    }
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
    e = cudaMalloc(&b->d_imgs, sizeof(ImgDesc) * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ta, sizeof(float) * std::max<size_t>(1, ta.size()));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tt, sizeof(float) * std::max<size_t>(1, tt.size()));
    for (int k = 0; k < b->n_lanes && e == cudaSuccess; ++k)
        e = cudaMalloc(&b->d_scratch[k], lane_ws[k]);
    if (e == cudaSuccess && !ta.empty())
        e = cudaMemcpy(b->d_ta, ta.data(), sizeof(float) * ta.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !tt.empty())
        e = cudaMemcpy(b->d_tt, tt.data(), sizeof(float) * tt.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = batch_apply_config(b);
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
    // finish what ran on the old pointers, then the tables and the graph
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = batch_apply_config(b);
    if (e != cudaSuccess) return cuda_check(e, "bf_batch_bind");
    b->bound = true;
    e = batch_build_graph(b);
    if (e != cudaSuccess) {
        b->bound = false;
        return cuda_check(e, "bf_batch_bind");
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

extern "C" bf_status bf_batch_config(const bf_batch *b, int r, int *shape, int *split) {
    if (!b) return fail(BF_EINVAL, "bf_batch_config: batch is NULL");
    if (r < 1 || r > kBatchTileMaxR)
        return fail(BF_EINVAL, "bf_batch_config: r must be in 1 .. 8 (larger half-widths run "
                               "the streaming sweeps)");
    if (shape) *shape = b->cfg_shape[r];
    if (split) *split = b->cfg_split[r];
    return BF_OK;
}

extern "C" bf_status bf_batch_set_config(bf_batch *b, int r, int shape, int split,
                                         cudaStream_t stream) {
    if (!b) return fail(BF_EINVAL, "bf_batch_set_config: batch is NULL");
    if (r < 1 || r > kBatchTileMaxR)
        return fail(BF_EINVAL, "bf_batch_set_config: r must be in 1 .. 8");
    if (!batch_shape_ok(r, shape))
        return fail(BF_EINVAL, "bf_batch_set_config: shape " + std::to_string(shape) +
                                   " is not available at r = " + std::to_string(r));
    if (split != 1 && split != 2 && split != 4)
        return fail(BF_EINVAL, "bf_batch_set_config: split must be 1, 2 or 4");
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_check(e, "bf_batch_set_config");
    b->cfg_shape[r] = shape;
    b->cfg_split[r] = split;
    e = batch_apply_config(b);
    if (e == cudaSuccess) e = batch_build_graph(b);
    return cuda_check(e, "bf_batch_set_config");
}

// Fastest of `reps` replays (one warm-up first): interference from outside
// only ever slows a replay down, so the minimum is the steadiest figure.
static cudaError_t batch_time(bf_batch *b, cudaStream_t stream, int reps, cudaEvent_t e0,
                              cudaEvent_t e1, float *ms) {
    cudaError_t e = cudaGraphLaunch(b->exec, stream);
    *ms = 1e30f;
    for (int k = 0; k < reps && e == cudaSuccess; ++k) {
        float t = 0.f;
        e = cudaEventRecord(e0, stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess) *ms = std::min(*ms, t);
    }
    return e;
}

// The same for the tiled images' launch alone (outside the graph, without
// the streaming images): the figure the per-bucket choices are made on, since
// one bucket's configuration moves the whole batch by about as much as the
// run-to-run spread of the streaming chains.
static cudaError_t batch_time_tiles(bf_batch *b, cudaStream_t stream, int reps, cudaEvent_t e0,
                                    cudaEvent_t e1, float *ms) {
    cudaError_t e = batch_launch_tiles(b, stream);
    *ms = 1e30f;
    for (int k = 0; k < reps && e == cudaSuccess; ++k) {
        float t = 0.f;
        e = cudaEventRecord(e0, stream);
        if (e == cudaSuccess) e = batch_launch_tiles(b, stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess) *ms = std::min(*ms, t);
    }
    return e;
}

// A candidate replaces the configuration in hand only when it is faster by
// more than this fraction, so that timing noise does not trade a plain
// configuration for one with more launches.
constexpr float kTuneMargin = 0.01f;

// Autotuner for a bound batch.  First, for each radius bucket of tiled
// images in turn (largest share of the tile work first), every tile shape the
// bucket has and every term split (1, 2, 4) with the other buckets as they
// stand, each timed on the tiled images' launch alone; then the persistent
// grid (1x or 2x the resident blocks) and the queue order (largest cost first
// or image order), each timed as the whole batch.  The result is kept in the
// batch's graph and reported.
extern "C" bf_status bf_batch_tune(bf_batch *b, cudaStream_t stream, int reps, int *grid_out,
                                   int *order_out, float *ms_out) {
    if (!b) return fail(BF_EINVAL, "bf_batch_tune: batch is NULL");
    if (!b->bound) return fail(BF_EINVAL, "bf_batch_tune: call bf_batch_bind first");
    if (reps < 1) reps = 3;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_check(e, "bf_batch_tune");
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    // buckets by their tile work (terms x pixels)
    double work[kBatchTileMaxR + 1] = {};
    for (const ImgDesc &d : b->h_imgs)
        if (d.r <= kBatchTileMaxR) work[d.r] += (double)d.n_terms * d.H * d.W;
    std::vector<int> buckets;
    for (int r = 1; r <= kBatchTileMaxR; ++r)
        if (work[r] > 0) buckets.push_back(r);
    std::stable_sort(buckets.begin(), buckets.end(), [&](int x, int y) { return work[x] > work[y]; });
    float best = 1e30f;
    const int treps = 2 * reps + 1;  // the tile launch is short: more samples
    if (e == cudaSuccess && b->n_tiles > 0) e = batch_time_tiles(b, stream, treps, e0, e1, &best);
    for (int r : buckets) {
        int best_shape = b->cfg_shape[r], best_split = b->cfg_split[r];
        for (int sh : {0, 1, 3}) {
            if (!batch_shape_ok(r, sh)) continue;
            for (int split : {1, 2, 4}) {
                if (e != cudaSuccess) break;
                if (sh == best_shape && split == best_split) continue;
                b->cfg_shape[r] = sh;
                b->cfg_split[r] = split;
                e = batch_apply_config(b);
                float ms = 0.f;
                if (e == cudaSuccess) e = batch_time_tiles(b, stream, treps, e0, e1, &ms);
                if (e == cudaSuccess && ms < best * (1.f - kTuneMargin)) {
                    best = ms;
                    best_shape = sh;
                    best_split = split;
                }
            }
        }
        b->cfg_shape[r] = best_shape;
        b->cfg_split[r] = best_split;
    }
    if (e == cudaSuccess) e = batch_apply_config(b);
    if (e == cudaSuccess) e = batch_build_graph(b);
    if (e == cudaSuccess) e = batch_time(b, stream, reps, e0, e1, &best);  // a fresh baseline
    int best_grid = b->grid, best_order = b->order;
    const int grids[2] = {std::min(b->resident, b->n_tiles),
                          std::min(2 * b->resident, b->n_tiles)};
    for (int order = 0; order < 2 && e == cudaSuccess; ++order) {
        for (int gi = 0; gi < 2 && e == cudaSuccess; ++gi) {
            b->order = order;
            e = batch_apply_config(b);
            b->grid = std::max(1, grids[gi]);
            if (e == cudaSuccess) e = batch_build_graph(b);
            float ms = 0.f;
            if (e == cudaSuccess) e = batch_time(b, stream, reps, e0, e1, &ms);
            if (e == cudaSuccess && ms < best * (1.f - kTuneMargin)) {
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
    e = batch_apply_config(b);
    b->grid = best_grid;
    if (e == cudaSuccess) e = batch_build_graph(b);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_check(e, "bf_batch_tune");
    if (grid_out) *grid_out = best_grid;
    if (order_out) *order_out = best_order;
    if (ms_out) *ms_out = best;
    return BF_OK;
}

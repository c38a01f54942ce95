// Unfused baseline: Algorithm 1 read literally, one term at a time, with the
// auxiliary images materialised in device memory (Section 2.2 describes the
// O(1) algorithm as: set up the auxiliary images, average each of them, then
// form the sums and the ratio of eq. (final-form)).
//
// Per term m, four kernels:
//   uf_gen    : A[p] = cos(w f), sin(w f), f cos(w f), f sin(w f)   (4 planes)
//   uf_vpass  : B = vertical 1-D filter of A (clamp-to-edge)
//   uf_hpass  : A = horizontal 1-D filter of B (clamp-to-edge)
//   uf_accum  : P += a cos(w f) A[2] + a sin(w f) A[3],
//               Q += a cos(w f) A[0] + a sin(w f) A[1]
// and once at the end uf_final: out = P / Q.  Every kernel is bound by device
// memory traffic; the 1-D passes stage a tile plus halo in shared memory and
// run the box cascade (any half-width r) or the Gaussian taps in place there.
#include <algorithm>

#include "bf_internal.h"
#include "bf_tile.cuh"

namespace bf {

namespace {

constexpr int kUfCols = 64;   // columns per vertical-pass block (one plane)
constexpr int kUfRowsV = 64;  // output rows per vertical-pass block
constexpr int kUfRowsH = 64;  // rows per horizontal-pass block
constexpr int kUfColsH = 64;  // output columns per horizontal-pass block

__global__ void uf_gen(const float *__restrict__ f, float *__restrict__ A, long long n, float tm) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = f[i];
    const float c = sin_turns(fmaf(tm, v, 0.25f));
    const float s = sin_turns(tm * v);
    A[i] = c;
    A[n + i] = s;
    A[2 * n + i] = v * c;
    A[3 * n + i] = v * s;
}

// In-place 1-D filter of a strided sequence a[0 .. n_in) in shared memory:
// box cascade of `passes` half-width-r boxes, or Gaussian taps of half-width R.
// Outputs land in a[0 .. n_in - 2 halo).
__device__ void filter_inplace(float *a, int stride, int n_in, int kind, int rad,
                               const float *__restrict__ w) {
    if (kind == 1) {
        int n = n_in;
        for (int pass = 0; pass < 3; ++pass) {
            const int nout = n - 2 * rad;
            float s = 0.f;
            for (int d = 0; d <= 2 * rad; ++d) s += a[d * stride];
            float prev = a[0];
            a[0] = s;
            for (int k = 1; k < nout; ++k) {
                const float nxt = a[(k + 2 * rad) * stride];
                const float cur = a[k * stride];
                s += nxt - prev;
                a[k * stride] = s;
                prev = cur;
            }
            n = nout;
        }
    } else {
        const int nout = n_in - 2 * rad;
        for (int k = 0; k < nout; ++k) {
            float acc = w[0] * a[k * stride];
            for (int d = 1; d <= 2 * rad; ++d) acc = fmaf(w[d], a[(k + d) * stride], acc);
            a[k * stride] = acc;
        }
    }
}

struct UfPass {
    int H, W, kind, rad, halo;
    BfTaps taps;
};

// grid: (ceil(W / kUfCols), ceil(H / kUfRowsV), 4 planes); block: kUfCols threads
__global__ void uf_vpass(const float *__restrict__ A, float *__restrict__ B,
                         const __grid_constant__ UfPass p) {
    extern __shared__ float sm[];
    const int H = p.H, W = p.W, halo = p.halo;
    const long long n = (long long)H * W;
    const int x = blockIdx.x * kUfCols + threadIdx.x;
    const int y0 = blockIdx.y * kUfRowsV;
    const float *src = A + blockIdx.z * n;
    float *dst = B + blockIdx.z * n;
    const int n_in = kUfRowsV + 2 * halo;
    const int xc = min(x, W - 1);
    for (int i = 0; i < n_in; ++i) {
        const int gy = min(max(y0 - halo + i, 0), H - 1);
        sm[i * kUfCols + threadIdx.x] = src[(long long)gy * W + xc];
    }
    filter_inplace(sm + threadIdx.x, kUfCols, n_in, p.kind, p.rad, p.taps.w);
    if (x < W)
        for (int i = 0; i < kUfRowsV && y0 + i < H; ++i)
            dst[(long long)(y0 + i) * W + x] = sm[i * kUfCols + threadIdx.x];
}

// grid: (ceil(W / kUfColsH), ceil(H / kUfRowsH), 4 planes); block: kUfRowsH threads
__global__ void uf_hpass(const float *__restrict__ B, float *__restrict__ A,
                         const __grid_constant__ UfPass p) {
    extern __shared__ float sm[];
    const int H = p.H, W = p.W, halo = p.halo;
    const long long n = (long long)H * W;
    const int x0 = blockIdx.x * kUfColsH;
    const int y0 = blockIdx.y * kUfRowsH;
    const float *src = B + blockIdx.z * n;
    float *dst = A + blockIdx.z * n;
    const int n_in = kUfColsH + 2 * halo;
    const int stride = n_in | 1;  // odd row stride: threads on rows hit distinct banks
    // cooperative coalesced load: consecutive threads take consecutive columns
    for (int r = 0; r < kUfRowsH; ++r) {
        const int gy = min(y0 + r, H - 1);
        for (int j = threadIdx.x; j < n_in; j += blockDim.x) {
            const int gx = min(max(x0 - halo + j, 0), W - 1);
            sm[r * stride + j] = src[(long long)gy * W + gx];
        }
    }
    __syncthreads();
    filter_inplace(sm + threadIdx.x * stride, 1, n_in, p.kind, p.rad, p.taps.w);
    __syncthreads();
    for (int r = 0; r < kUfRowsH; ++r) {
        const int gy = y0 + r;
        if (gy >= H) break;
        for (int j = threadIdx.x; j < kUfColsH; j += blockDim.x)
            if (x0 + j < W) dst[(long long)gy * W + x0 + j] = sm[r * stride + j];
    }
}

__global__ void uf_accum(const float *__restrict__ f, const float *__restrict__ A,
                         float *__restrict__ P, float *__restrict__ Q, long long n, float am,
                         float tm, int first) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = f[i];
    const float c = am * sin_turns(fmaf(tm, v, 0.25f));
    const float s = am * sin_turns(tm * v);
    float p = first ? 0.f : P[i];
    float q = first ? 0.f : Q[i];
    p = fmaf(c, A[2 * n + i], p);
    p = fmaf(s, A[3 * n + i], p);
    q = fmaf(c, A[i], q);
    q = fmaf(s, A[n + i], q);
    P[i] = p;
    Q[i] = q;
}

__global__ void uf_final(const float *__restrict__ P, const float *__restrict__ Q,
                         float *__restrict__ out, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = P[i] / Q[i];
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t unfused_workspace(int H, int W) {
    const size_t n = (size_t)H * (size_t)W;
    return 2 * align256(4 * n * sizeof(float)) + 2 * align256(n * sizeof(float)) + 256;
}

cudaError_t launch_unfused(const bf_plan *pl, const float *in, float *out, int H, int W,
                           void *ws, cudaStream_t s) {
    const long long n = (long long)H * W;
    char *base = reinterpret_cast<char *>(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    float *A = reinterpret_cast<float *>(base);
    float *B = reinterpret_cast<float *>(base + align256(4 * n * sizeof(float)));
    float *P = reinterpret_cast<float *>(base + 2 * align256(4 * n * sizeof(float)));
    float *Q = reinterpret_cast<float *>(base + 2 * align256(4 * n * sizeof(float)) +
                                         align256(n * sizeof(float)));
    UfPass up;
    up.H = H;
    up.W = W;
    up.kind = pl->kind == BF_SPATIAL_BOX_ITER ? 1 : 0;
    up.rad = pl->kind == BF_SPATIAL_BOX_ITER ? pl->r_box : pl->R;
    up.halo = pl->R;
    fill_taps(pl, &up.taps);
    const size_t smv = sizeof(float) * (size_t)(kUfRowsV + 2 * up.halo) * kUfCols;
    const size_t smh = sizeof(float) * (size_t)kUfRowsH * ((kUfColsH + 2 * up.halo) | 1);
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        e = cudaFuncSetAttribute(uf_vpass, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(uf_hpass, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    if (smv > 227 * 1024 || smh > 227 * 1024) return cudaErrorInvalidValue;
    const int tpb = 256;
    const unsigned nb = (unsigned)((n + tpb - 1) / tpb);
    dim3 gv((W + kUfCols - 1) / kUfCols, (H + kUfRowsV - 1) / kUfRowsV, 4);
    dim3 gh((W + kUfColsH - 1) / kUfColsH, (H + kUfRowsH - 1) / kUfRowsH, 4);
    const int nt = (int)pl->a32.size();
    for (int m = 0; m < nt; ++m) {
        uf_gen<<<nb, tpb, 0, s>>>(in, A, n, pl->turns32[m]);
        uf_vpass<<<gv, kUfCols, smv, s>>>(A, B, up);
        uf_hpass<<<gh, kUfRowsH, smh, s>>>(B, A, up);
        uf_accum<<<nb, tpb, 0, s>>>(in, A, P, Q, n, pl->a32[m], pl->turns32[m], m == 0);
    }
    uf_final<<<nb, tpb, 0, s>>>(P, Q, out, n);
    return cudaGetLastError();
}

}  // namespace bf

// Forward filter for the 3-pass box at large half-widths r (support 3r > 24).
//
// A tile plus a 3r halo no longer fits on chip, so the separable filter is
// run as two streaming sweeps per term, with the term's filtered auxiliary
// images passing through device memory once (small enough to stay in L2
// between the two sweeps for images up to about 2048 x 2048):
//
//   lr_vert : one thread per image column and plane, walking down a band of
//             rows (f loaded a few rows ahead).  The four auxiliary
//             images of the term (cos, sin, f cos, f sin of omega f,
//             Section 2.3) are generated on the fly and filtered by the three
//             cascaded boxes with running sums; written transposed
//             (column-major) so that the second sweep reads coalesced.
//   lr_horz : one thread per image row and plane, walking along a band of columns of the
//             transposed planes (loads issued a few steps ahead): the same
//             three cascaded boxes horizontally, then the per-pixel combine of
//             eq. (final-form), accumulated per plane (column-major).
//   lr_final: out = P / Q, with P and Q the sums of the plane accumulators,
//             transposed back to row-major.
//
// Running sums with one history buffer.  Box k of the cascade at position q
// needs its input at q + r and q - r - 1.  Keeping one running sum per
// position that a later box needs (three for the first box, two for the
// second, one for the third, spaced L = 2r + 1 apart) makes every update read
// only the raw input at the four positions e, e - L, e - 2L, e - 3L: the
// newest is generated (or loaded), the other three come from a ring of the
// last 3L + 1 inputs in shared memory.  Each running sum is a plain sliding
// sum (add the incoming, subtract the outgoing), so rounding grows like the
// usual running sum, and the half-width r is a run-time value.  The sums start
// at zero 3r positions before the first output with the input taken as zero
// before that point, so the first 6r steps of a band are warm-up.
#include <algorithm>

#include "bf_internal.h"
#include "bf_tile.cuh"

namespace bf {

namespace {

constexpr int kLvCols = 32;   // columns per lr_vert block; one warp per plane
constexpr int kLvStage = 8;   // lr_vert: output rows staged before a transposed flush
constexpr int kLhRows = 32;   // rows per lr_horz block; one warp per plane

struct LrParams {
    const void *in;
    long long in_stride;  // elements
    int dtype, C, ch;
    int H, W, r;
    int band_h, band_w;
    float a, t;           // weight and turns per gray level of this term
    float *Vt;            // [4][W][H]: vertically filtered planes, column-major
    float *Acc;           // [4][W][H]: sum over terms of a cos|sin(w f(x)) W[plane](x)
    int first;
};

__device__ __forceinline__ float load_f(const LrParams &p, int y, int x) {
    const long long off = (long long)y * p.in_stride + (long long)x * p.C + p.ch;
    if (p.dtype == 0) return __ldg(reinterpret_cast<const float *>(p.in) + off);
    return (float)__ldg(reinterpret_cast<const uint8_t *>(p.in) + off);
}

// Plane q of the auxiliary images at one pixel value fv:
// q = 0: cos, 1: sin, 2: f cos, 3: f sin (cos(t) = sin(t + quarter turn)).
__device__ __forceinline__ float aux_plane(int q, float tm, float fv) {
    const float v = sin_turns(fmaf(tm, fv, (q & 1) ? 0.f : 0.25f));
    return q >= 2 ? v * fv : v;
}

// Ring of the last 3L + 1 input values of one running-sum stream per thread,
// in shared memory, [slot][lane] so that a warp's accesses are conflict-free.
struct Ring {
    float *base;
    int n;      // slots (3L + 1)
    int head;   // slot of the newest value
    __device__ __forceinline__ void push(float v, int lane) {
        head = head + 1 == n ? 0 : head + 1;
        base[head * 32 + lane] = v;
    }
    // value k*L positions behind the newest (k = 1..3)
    __device__ __forceinline__ float back(int off, int lane) const {
        int s = head - off;
        s = s < 0 ? s + n : s;
        return base[s * 32 + lane];
    }
};

template <int DT>
__device__ __forceinline__ float load_px(const LrParams &p, int y, int x) {
    const long long off = (long long)y * p.in_stride + (long long)x * p.C + p.ch;
    if constexpr (DT == 0) return __ldg(reinterpret_cast<const float *>(p.in) + off);
    else return (float)__ldg(reinterpret_cast<const uint8_t *>(p.in) + off);
}

constexpr int kChunk = 16;  // steps whose global loads are issued together

// grid: (ceil(W / kLvCols), bands); block: 4 warps (warp q = plane q), lanes =
// columns.  Dynamic smem: one ring of 3L + 1 generated values per thread.
template <int DT>
__global__ void __launch_bounds__(4 * kLvCols) lr_vert(const __grid_constant__ LrParams p) {
    extern __shared__ float lv_sm[];
    const int lane = threadIdx.x & 31;
    const int q = threadIdx.x >> 5;
    const int xb = blockIdx.x * kLvCols;
    const int xc = min(xb + lane, p.W - 1);
    const float tm = p.t;
    const int y0 = blockIdx.y * p.band_h;
    const int y1 = min(y0 + p.band_h, p.H);
    const int r = p.r, L = 2 * r + 1;
    const int p0 = y0 - 3 * r;  // first position whose input is taken as real
    const int e_end = y1 + 3 * r;
    Ring ring{lv_sm + (size_t)q * (3 * L + 1) * 32, 3 * L + 1, 0};
    for (int k = 0; k < ring.n; ++k) ring.base[k * 32 + lane] = 0.f;  // zero input before p0
    float s1a = 0.f, s1b = 0.f, s1c = 0.f, s2a = 0.f, s2b = 0.f, s3 = 0.f;
    float *dst_col = p.Vt + (size_t)q * p.W * p.H + (size_t)(xb + lane) * p.H;
    const bool col_ok = xb + lane < p.W;
    float stage[kLvStage];
    // f of the next chunk of rows is loaded while the current one is used
    float cur[kChunk], nxt[kChunk];
#pragma unroll
    for (int d = 0; d < kChunk; ++d) cur[d] = load_px<DT>(p, min(max(p0 + d, 0), p.H - 1), xc);
    for (int e0 = p0; e0 < e_end; e0 += kChunk) {
#pragma unroll
        for (int d = 0; d < kChunk; ++d)
            nxt[d] = load_px<DT>(p, min(max(e0 + kChunk + d, 0), p.H - 1), xc);
#pragma unroll
        for (int d = 0; d < kChunk; ++d) {
            const int e = e0 + d;
            if (e < e_end) {
                const float x0 = aux_plane(q, tm, cur[d]);
                const float x1 = ring.back(L - 1, lane);      // position e - L
                const float x2 = ring.back(2 * L - 1, lane);  // e - 2L
                const float x3 = ring.back(3 * L - 1, lane);  // e - 3L
                ring.push(x0, lane);
                s1a += x0 - x1;
                s1b += x1 - x2;
                s1c += x2 - x3;
                s2a += s1a - s1b;
                s2b += s1b - s1c;
                s3 += s2a - s2b;
                const int t = e - 3 * r;  // output row of this step
                if (t >= y0) {
                    const int j = (t - y0) & (kLvStage - 1);
#pragma unroll
                    for (int jj = 0; jj < kLvStage; ++jj)
                        if (jj == j) stage[jj] = s3;
                    if ((j == kLvStage - 1 || t == y1 - 1) && col_ok) {
                        const int yb = t - j;
#pragma unroll
                        for (int jj = 0; jj < kLvStage; ++jj)
                            if (jj <= j) dst_col[yb + jj] = stage[jj];
                    }
                }
            }
        }
#pragma unroll
        for (int d = 0; d < kChunk; ++d) cur[d] = nxt[d];
    }
}

// grid: (ceil(H / kLhRows), bands along x); block: 4 warps (warp q = plane q),
// lanes = rows.  Dynamic smem: one ring of 3L + 1 values per thread.
template <int DT>
__global__ void __launch_bounds__(4 * kLhRows) lr_horz(const __grid_constant__ LrParams p) {
    extern __shared__ float lh_sm[];
    const int lane = threadIdx.x & 31;
    const int q = threadIdx.x >> 5;
    const int y = blockIdx.x * kLhRows + lane;
    const int yc = min(y, p.H - 1);
    const int x0 = blockIdx.y * p.band_w;
    const int x1 = min(x0 + p.band_w, p.W);
    const int r = p.r, L = 2 * r + 1;
    const int p0 = x0 - 3 * r;
    const size_t plane = (size_t)p.W * p.H;
    const float *V = p.Vt + q * plane + yc;
    float *A = p.Acc + q * plane;
    const int e_end = x1 + 3 * r;
    Ring ring{lh_sm + (size_t)q * (3 * L + 1) * 32, 3 * L + 1, 0};
    for (int k = 0; k < ring.n; ++k) ring.base[k * 32 + lane] = 0.f;
    float s1a = 0.f, s1b = 0.f, s1c = 0.f, s2a = 0.f, s2b = 0.f, s3 = 0.f;
    const float ph0 = (q & 1) ? 0.f : 0.25f;  // cos for planes 0 and 2, sin for 1 and 3
    // the plane at the positions of the next chunk, and the pixel values and
    // running accumulators of the chunk's outputs, loaded one chunk ahead
    float cv[kChunk], cf[kChunk], ca[kChunk];
    float nv[kChunk], nf[kChunk], na[kChunk];
    auto fetch = [&](int eb, float (&v)[kChunk], float (&f)[kChunk], float (&a)[kChunk]) {
#pragma unroll
        for (int d = 0; d < kChunk; ++d) {
            const int e = eb + d;
            v[d] = __ldg(V + (size_t)min(max(e, 0), p.W - 1) * p.H);
            const int t = min(max(e - 3 * r, 0), p.W - 1);
            f[d] = load_px<DT>(p, yc, t);
            a[d] = p.first ? 0.f : A[(size_t)t * p.H + yc];
        }
    };
    fetch(p0, cv, cf, ca);
    for (int e0 = p0; e0 < e_end; e0 += kChunk) {
        fetch(e0 + kChunk, nv, nf, na);
#pragma unroll
        for (int d = 0; d < kChunk; ++d) {
            const int e = e0 + d;
            if (e < e_end) {
                const float xin = cv[d];
                const float x1v = ring.back(L - 1, lane);
                const float x2v = ring.back(2 * L - 1, lane);
                const float x3v = ring.back(3 * L - 1, lane);
                ring.push(xin, lane);
                s1a += xin - x1v;
                s1b += x1v - x2v;
                s1c += x2v - x3v;
                s2a += s1a - s1b;
                s2b += s1b - s1c;
                s3 += s2a - s2b;
                const int t = e - 3 * r;  // output column of this step
                if (t >= x0 && y < p.H) {
                    const float coef = p.a * sin_turns(fmaf(p.t, cf[d], ph0));
                    A[(size_t)t * p.H + y] = fmaf(coef, s3, ca[d]);
                }
            }
        }
#pragma unroll
        for (int d = 0; d < kChunk; ++d) {
            cv[d] = nv[d];
            cf[d] = nf[d];
            ca[d] = na[d];
        }
    }
}

// out = (A2 + A3) / (A0 + A1) (numerator: f cos, f sin planes; normaliser:
// cos, sin planes), column-major -> row-major through a 32 x 33 shared tile.
// grid: (ceil(W / 32), ceil(H / 32)); block: (32, 8)
__global__ void lr_final(const float *__restrict__ Acc, float *__restrict__ out,
                         float *__restrict__ q_out, int H, int W, int C, int ch, float q_scale) {
    __shared__ float tp[32][33];
    __shared__ float tq[32][33];
    const size_t plane = (size_t)W * H;
    const int xb = blockIdx.x * 32, yb = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int x = xb + i, y = yb + threadIdx.x;
        if (x < W && y < H) {
            const size_t o = (size_t)x * H + y;
            tq[i][threadIdx.x] = Acc[o] + Acc[plane + o];
            tp[i][threadIdx.x] = Acc[2 * plane + o] + Acc[3 * plane + o];
        }
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int y = yb + i, x = xb + threadIdx.x;
        if (x < W && y < H) {
            const float q = tq[threadIdx.x][i];
            const size_t o = ((size_t)y * W + x) * C + ch;
            out[o] = tp[threadIdx.x][i] / q;
            if (q_out) q_out[o] = q * q_scale;
        }
    }
}

}  // namespace

size_t large_workspace(int H, int W) {
    return (size_t)8 * (size_t)H * (size_t)W * sizeof(float) + 256;
}

cudaError_t launch_large_box(const bf_plan *pl, const BfImage &img, void *ws, cudaStream_t s) {
    const int H = img.H, W = img.W;
    char *base = reinterpret_cast<char *>(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    LrParams p;
    p.in = img.in;
    p.in_stride = img.in_row_stride;
    p.dtype = img.dtype;
    p.C = img.C;
    p.H = H;
    p.W = W;
    p.r = pl->r_box;
    p.Vt = reinterpret_cast<float *>(base);
    p.Acc = p.Vt + (size_t)4 * H * W;
    // bands: long enough to amortise the 6r warm-up, short enough to fill the GPU
    p.band_h = std::max(256, 8 * p.r);
    p.band_w = std::max(256, 8 * p.r);
    const int nbh = (H + p.band_h - 1) / p.band_h;
    const int nbw = (W + p.band_w - 1) / p.band_w;
    // one ring of 3L + 1 values per thread, 128 threads per block
    const size_t sm_ring = sizeof(float) * (size_t)4 * 32 * (3 * (2 * p.r + 1) + 1);
    if (sm_ring > 227 * 1024) return cudaErrorInvalidValue;
    auto kv = img.dtype == 0 ? lr_vert<0> : lr_vert<1>;
    auto kh = img.dtype == 0 ? lr_horz<0> : lr_horz<1>;
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        for (auto k : {lr_vert<0>, lr_vert<1>, lr_horz<0>, lr_horz<1>}) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
            if (e != cudaSuccess) return e;
        }
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    const int nt = (int)pl->a32.size();
    for (int ch = 0; ch < img.C; ++ch) {
        p.ch = ch;
        for (int m = 0; m < nt; ++m) {
            p.a = pl->a32[m];
            p.t = pl->turns32[m];
            p.first = m == 0;
            dim3 gv((W + kLvCols - 1) / kLvCols, nbh);
            kv<<<gv, 4 * kLvCols, sm_ring, s>>>(p);
            dim3 gh((H + kLhRows - 1) / kLhRows, nbw);
            kh<<<gh, 4 * kLhRows, sm_ring, s>>>(p);
        }
        dim3 gf((W + 31) / 32, (H + 31) / 32);
        lr_final<<<gf, dim3(32, 8), 0, s>>>(p.Acc, img.out, img.q_out, H, W, img.C, ch,
                                            img.q_scale);
    }
    return cudaGetLastError();
}

}  // namespace bf

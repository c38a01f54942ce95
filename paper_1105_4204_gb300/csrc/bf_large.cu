// Forward filter for the 3-pass box at large half-widths r (support 3r > 24).
//
// A tile plus a 3r halo no longer fits on chip, so the separable filter is
// run as two streaming sweeps per term, with the term's filtered auxiliary
// images passing through device memory once (small enough to stay in L2
// between the two sweeps for images up to about 2048 x 2048):
//
//   lr_vert : one thread per image column and term (four terms per block,
//             sharing a ring of f), walking down a band of rows (f loaded a
//             few rows ahead).  The four auxiliary
//             images of the term (cos, sin, f cos, f sin of omega f,
//             Section 2.3) are generated on the fly and filtered by the three
//             cascaded boxes with running sums; written transposed
//             (column-major) so that the second sweep reads coalesced.
//   lr_horz : one thread per image row and plane pair, walking along a band
//             of columns of the transposed planes (loads issued a chunk
//             ahead; the trailing inputs are read again from L2 instead of
//             being kept on chip): the same three cascaded boxes horizontally
//             on the (cos, sin) or the (f cos, f sin) pair, then the
//             per-pixel combine of eq. (final-form) into Q or P.
//   lr_final: out = P / Q, transposed back to row-major.
//
// Running sums without per-pass history.  Box k of the cascade at position q
// needs its input at q + r and q - r - 1.  Keeping one running sum per
// position that a later box needs (three for the first box, two for the
// second, one for the third, spaced L = 2r + 1 apart) makes every update read
// only the raw input at the four positions e, e - L, e - 2L, e - 3L: the
// newest is generated (or loaded); the other three come from a shared-memory
// ring of f, the planes being regenerated (lr_vert), or are read again from
// the transposed planes in L2 (lr_horz).  Each running sum is a plain sliding
// sum (add the incoming, subtract the outgoing), so rounding grows like the
// usual running sum, and the half-width r is a run-time value.  The sums start
// at zero 3r positions before the first output with the input taken as zero
// before that point, so the first 6r steps of a band are warm-up.
#include <algorithm>
#include <type_traits>

#include "bf_internal.h"
#include "bf_tile.cuh"

namespace bf {

namespace {


struct LrParams {
    const void *in;       // first pixel of the plane being filtered
    long long in_stride;  // elements between rows
    int dtype, in_px;     // element type; elements between adjacent pixels
    int H, W, r;
    int band_h, band_w;
    float a, t;           // lr_horz: weight and turns per gray level of its term
    int slot;             // lr_horz: which of lr_vert's term slots it reads
    int n_terms;          // lr_vert: terms in this group (<= 4)
    float tv[4];          // lr_vert: turns per gray level of the group's terms
    int Hp;               // column length of the column-major arrays (H rounded up to 8)
    float *Vt;            // [4 terms][4 planes][W][Hp]: vertically filtered planes, column-major
    float *Acc;           // [2][W][Hp]: Q and P, column-major
    float *ft;            // [W][Hp]: the channel's f, column-major
    int first;
};

// Power-of-two size of lr_vert's shared f ring: the 3L + 1 values a stream
// needs, plus slack for the warps sharing it to be up to two chunks apart
// (they meet at a barrier every chunk) without overwriting a value another
// warp still has to read.
__host__ __device__ __forceinline__ int ring_size(int r) {
    int n = 1;
    while (n < 3 * (2 * r + 1) + 1 + 16) n <<= 1;
    return n;
}

template <int DT>
__device__ __forceinline__ float load_px(const LrParams &p, int y, int x) {
    const long long off = (long long)y * p.in_stride + (long long)x * p.in_px;
    if constexpr (DT == 0) return __ldg(reinterpret_cast<const float *>(p.in) + off);
    else return (float)__ldg(reinterpret_cast<const uint8_t *>(p.in) + off);
}

constexpr int kVCols = 64;    // lr_vert: columns per block
constexpr int kVG = 4;        // lr_vert: terms per block (they share the f ring)
constexpr int kChunk = 8;     // lr_vert: steps between barriers / whose loads are issued together
constexpr int kChunkH = 16;   // lr_horz: steps whose loads are issued together, one chunk ahead

// The four auxiliary planes of one pixel value (cos, sin, f cos, f sin).
__device__ __forceinline__ void aux4(float tm, float fv, float (&x)[4]) {
    float r = tm * fv;
    r = r - rintf(r);
    float sn, cs;
    __sincosf(kTwoPi * r, &sn, &cs);
    x[0] = cs;
    x[1] = sn;
    x[2] = fv * cs;
    x[3] = fv * sn;
}

// grid: (ceil(W / kVCols), bands); block: kVCols x kVG threads, thread
// (column, term g) computes the four planes of term g for one column.  The
// kVG terms share one ring of the last ring_size(r) values of f per column
// (every thread writes the same value into it; a barrier per chunk keeps the
// warps within kChunk steps of each other, far less than the ring's slack).
// Chunks are aligned so that step d of a chunk produces output row
// 8k + d of the band: the eight outputs of a chunk stay in registers and
// leave as two 16-byte stores per plane.  Dynamic smem: the f ring.
template <int DT>
__global__ void __launch_bounds__(kVCols * kVG) lr_vert(const __grid_constant__ LrParams p) {
    extern __shared__ float lv_sm[];
    const int tid = threadIdx.x;
    const int col = tid % kVCols;
    const int g = tid / kVCols;
    const int xb = blockIdx.x * kVCols;
    const int xc = min(xb + col, p.W - 1);
    const bool term_ok = g < p.n_terms;
    const float tm = p.tv[g];
    const int y0 = blockIdx.y * p.band_h;
    const int y1 = min(y0 + p.band_h, p.H);
    const int r = p.r, L = 2 * r + 1;
    const int p0 = y0 - 3 * r;  // inputs before p0 count as zero
    const int e_end = y1 + 3 * r;
    // first step: output row y0 falls on d = 0 of a chunk, and e_s <= p0
    const int e_s = p0 + 6 * r - kChunk * ((6 * r + kChunk - 1) / kChunk);
    const int RS = ring_size(r), M = RS - 1;
    float *ring = lv_sm + col;  // slot k at ring[k * kVCols]
    const bool col_ok = xb + col < p.W && term_ok;
    const size_t plane = (size_t)p.W * p.Hp;
    float *dst = p.Vt + (size_t)g * 4 * plane + (size_t)(xb + col) * p.Hp;
    float s1[4][3], s2[4][2], s3[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        s1[q][0] = s1[q][1] = s1[q][2] = 0.f;
        s2[q][0] = s2[q][1] = 0.f;
        s3[q] = 0.f;
    }
    float cur[kChunk], nxt[kChunk];
#pragma unroll
    for (int d = 0; d < kChunk; ++d) cur[d] = load_px<DT>(p, min(max(e_s + d, 0), p.H - 1), xc);
    float st[4][kChunk];
    // one step; CHECKED covers steps before p0 + 3L (inputs before p0 are
    // zero) and the band's last chunk
    auto step = [&](int e, int d, auto checked) {
        constexpr bool CHECKED = decltype(checked)::value;
        const float fv = cur[d];
        ring[(e & M) * kVCols] = fv;
        float x0[4], x1[4], x2[4], x3[4];
        aux4(tm, fv, x0);
        if (!CHECKED) {
            aux4(tm, ring[((e - L) & M) * kVCols], x1);
            aux4(tm, ring[((e - 2 * L) & M) * kVCols], x2);
            aux4(tm, ring[((e - 3 * L) & M) * kVCols], x3);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) x1[q] = x2[q] = x3[q] = 0.f;
            if (e < p0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) x0[q] = 0.f;
            }
            if (e >= p0 + L) aux4(tm, ring[((e - L) & M) * kVCols], x1);
            if (e >= p0 + 2 * L) aux4(tm, ring[((e - 2 * L) & M) * kVCols], x2);
            if (e >= p0 + 3 * L) aux4(tm, ring[((e - 3 * L) & M) * kVCols], x3);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            s1[q][0] += x0[q] - x1[q];
            s1[q][1] += x1[q] - x2[q];
            s1[q][2] += x2[q] - x3[q];
            s2[q][0] += s1[q][0] - s1[q][1];
            s2[q][1] += s1[q][1] - s1[q][2];
            s3[q] += s2[q][0] - s2[q][1];
            st[q][d] = s3[q];
        }
    };
    for (int e0 = e_s; e0 < e_end; e0 += kChunk) {
        __syncthreads();  // bounds the skew between the warps sharing the ring
#pragma unroll
        for (int d = 0; d < kChunk; ++d)
            nxt[d] = load_px<DT>(p, min(max(e0 + kChunk + d, 0), p.H - 1), xc);
        const int tb = e0 - 3 * r;  // output row of step d = 0 (tb - y0 is a multiple of 8)
        const bool fast = e0 >= p0 + 3 * L && e0 + kChunk <= e_end;  // uniform
        if (fast) {
#pragma unroll
            for (int d = 0; d < kChunk; ++d) step(e0 + d, d, std::false_type{});
        } else {
#pragma unroll
            for (int d = 0; d < kChunk; ++d)
                if (e0 + d < e_end) step(e0 + d, d, std::true_type{});
        }
        if (col_ok && tb >= y0) {
            if (tb + kChunk <= y1) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float4 *d4 = reinterpret_cast<float4 *>(dst + q * plane + tb);
                    d4[0] = make_float4(st[q][0], st[q][1], st[q][2], st[q][3]);
                    d4[1] = make_float4(st[q][4], st[q][5], st[q][6], st[q][7]);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int d = 0; d < kChunk; ++d)
                        if (tb + d < y1) dst[q * plane + tb + d] = st[q][d];
            }
        }
#pragma unroll
        for (int d = 0; d < kChunk; ++d) cur[d] = nxt[d];
    }
}

// f of one channel, row-major -> column-major (32 x 33 shared tile).
// grid: (ceil(W / 32), ceil(H / 32)); block: (32, 8)
template <int DT>
__global__ void lr_transpose(const __grid_constant__ LrParams p) {
    __shared__ float tile[32][33];
    const int xb = blockIdx.x * 32, yb = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int y = yb + i, x = xb + threadIdx.x;
        if (x < p.W && y < p.H) tile[i][threadIdx.x] = load_px<DT>(p, y, x);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int x = xb + i, y = yb + threadIdx.x;
        if (x < p.W && y < p.H) p.ft[(size_t)x * p.Hp + y] = tile[threadIdx.x][i];
    }
}

// grid: (ceil(H / 32), bands along x, 2); block: 64 threads = two warps of
// 32 rows each, lanes = rows.  blockIdx.z = 0: the (cos, sin) planes,
// accumulated into Q; blockIdx.z = 1: the (f cos, f sin) planes,
// accumulated into P.  Both planes of a pair share the pixel's sincos and
// one accumulator.  The inputs at e - L, e - 2L, e - 3L are read again from
// the transposed planes (L2) rather than kept, so no shared memory limits
// the number of resident warps.
constexpr int kChunkG = 8;
__global__ void __launch_bounds__(64) lr_horz(const __grid_constant__ LrParams p) {
    const int lane = threadIdx.x & 31;
    const int pr = blockIdx.z;  // 0: Q pair, 1: P pair
    const int y = (blockIdx.x * 2 + (threadIdx.x >> 5)) * 32 + lane;
    const int yc = min(y, p.H - 1);
    const int x0 = blockIdx.y * p.band_w;
    const int x1 = min(x0 + p.band_w, p.W);
    const int r = p.r, L = 2 * r + 1;
    const int p0 = x0 - 3 * r;
    const size_t plane = (size_t)p.W * p.Hp;
    const float *Vc = p.Vt + (size_t)p.slot * 4 * plane + (size_t)(2 * pr) * plane + yc;
    const float *Vs = Vc + plane;
    const float *F = p.ft + yc;
    float *A = p.Acc + (size_t)pr * plane + yc;
    const int e_end = x1 + 3 * r;
    const float am = p.a, tm = p.t;
    const bool row_ok = y < p.H;
    const bool first = p.first;
    float c1a = 0.f, c1b = 0.f, c1c = 0.f, c2a = 0.f, c2b = 0.f, c3 = 0.f;
    float z1a = 0.f, z1b = 0.f, z1c = 0.f, z2a = 0.f, z2b = 0.f, z3 = 0.f;
    // per chunk: both planes at e, e-L, e-2L, e-3L (0 before p0), and at the
    // chunk's outputs the pixel value and the pair's running accumulator
    float cv[kChunkG][8], cf[kChunkG], ca[kChunkG];
    float nv[kChunkG][8], nf[kChunkG], na[kChunkG];
    auto fetch = [&](int eb, float (&v)[kChunkG][8], float (&f)[kChunkG], float (&a)[kChunkG]) {
#pragma unroll
        for (int d = 0; d < kChunkG; ++d) {
            const int e = eb + d;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int pos = e - k * L;
                const size_t o = (size_t)min(max(pos, 0), p.W - 1) * p.Hp;
                const bool ok = pos >= p0;
                v[d][2 * k] = ok ? __ldg(Vc + o) : 0.f;
                v[d][2 * k + 1] = ok ? __ldg(Vs + o) : 0.f;
            }
            const size_t t = (size_t)min(max(e - 3 * r, 0), p.W - 1) * p.Hp;
            f[d] = __ldg(F + t);
            a[d] = first ? 0.f : A[t];
        }
    };
    fetch(p0, cv, cf, ca);
    for (int e0 = p0; e0 < e_end; e0 += kChunkG) {
        fetch(e0 + kChunkG, nv, nf, na);
        const bool full = e0 + kChunkG <= e_end && e0 - 3 * r >= x0;  // uniform
#pragma unroll
        for (int d = 0; d < kChunkG; ++d) {
            const int e = e0 + d;
            if (!full && e >= e_end) break;
            const float *v = cv[d];
            c1a += v[0] - v[2];
            c1b += v[2] - v[4];
            c1c += v[4] - v[6];
            c2a += c1a - c1b;
            c2b += c1b - c1c;
            c3 += c2a - c2b;
            z1a += v[1] - v[3];
            z1b += v[3] - v[5];
            z1c += v[5] - v[7];
            z2a += z1a - z1b;
            z2b += z1b - z1c;
            z3 += z2a - z2b;
            const int t = e - 3 * r;  // output column of this step
            if (full ? row_ok : (t >= x0 && row_ok)) {
                float rr = tm * cf[d];
                rr = rr - rintf(rr);
                float sn, cs;
                __sincosf(kTwoPi * rr, &sn, &cs);
                A[(size_t)t * p.Hp] = fmaf(am * cs, c3, fmaf(am * sn, z3, ca[d]));
            }
        }
#pragma unroll
        for (int d = 0; d < kChunkG; ++d) {
#pragma unroll
            for (int k = 0; k < 8; ++k) cv[d][k] = nv[d][k];
            cf[d] = nf[d];
            ca[d] = na[d];
        }
    }
}

// out = P / Q (accumulator 1 / accumulator 0), column-major -> row-major
// through a 32 x 33 shared tile.
// grid: (ceil(W / 32), ceil(H / 32)); block: (32, 8)
__global__ void lr_final(const float *__restrict__ Acc, float *__restrict__ out,
                         float *__restrict__ q_out, int H, int W, int Hp, int out_px,
                         float q_scale) {
    __shared__ float tp[32][33];
    __shared__ float tq[32][33];
    const size_t plane = (size_t)W * Hp;
    const int xb = blockIdx.x * 32, yb = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int x = xb + i, y = yb + threadIdx.x;
        if (x < W && y < H) {
            const size_t o = (size_t)x * Hp + y;
            tq[i][threadIdx.x] = Acc[o];
            tp[i][threadIdx.x] = Acc[plane + o];
        }
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int y = yb + i, x = xb + threadIdx.x;
        if (x < W && y < H) {
            const float q = tq[threadIdx.x][i];
            const size_t o = ((size_t)y * W + x) * out_px;
            out[o] = tp[threadIdx.x][i] / q;
            if (q_out) q_out[o] = q * q_scale;
        }
    }
}

}  // namespace

size_t large_workspace(int H, int W) {
    const size_t Hp = ((size_t)H + 7) / 8 * 8;
    return (size_t)(4 * kVG + 3) * Hp * (size_t)W * sizeof(float) + 256;
}

cudaError_t launch_large_box(const bf_plan *pl, const BfImage &img, void *ws, cudaStream_t s) {
    const int H = img.H, W = img.W;
    char *base = reinterpret_cast<char *>(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    LrParams p{};
    p.in_stride = img.in_row_stride;
    p.dtype = img.dtype;
    p.in_px = img.in_px;
    p.H = H;
    p.W = W;
    p.Hp = (H + 7) / 8 * 8;
    p.r = pl->r_box;
    p.Vt = reinterpret_cast<float *>(base);
    p.Acc = p.Vt + (size_t)4 * kVG * p.Hp * W;
    p.ft = p.Acc + (size_t)2 * p.Hp * W;
    // bands (multiples of 8 rows): long enough to amortise the 6r warm-up,
    // short enough to fill the GPU
    p.band_h = std::max(256, 8 * p.r);
    p.band_w = std::max(256, 8 * p.r);
    const int nbh = (H + p.band_h - 1) / p.band_h;
    const int nbw = (W + p.band_w - 1) / p.band_w;
    const int RS = ring_size(p.r);
    const size_t sm_v = sizeof(float) * (size_t)kVCols * RS;
    if (sm_v > 227 * 1024) return cudaErrorInvalidValue;
    auto kv = img.dtype == 0 ? lr_vert<0> : lr_vert<1>;
    auto kt = img.dtype == 0 ? lr_transpose<0> : lr_transpose<1>;
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        for (auto k : {lr_vert<0>, lr_vert<1>}) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
            if (e != cudaSuccess) return e;
        }
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    const int nt = (int)pl->a32.size();
    const int esz = img.dtype == 0 ? 4 : 1;
    for (int ch = 0; ch < img.C; ++ch) {
        p.in = reinterpret_cast<const char *>(img.in) + (long long)ch * img.in_z * esz;
        dim3 gt((W + 31) / 32, (H + 31) / 32);
        kt<<<gt, dim3(32, 8), 0, s>>>(p);
        for (int m0 = 0; m0 < nt; m0 += kVG) {
            p.n_terms = std::min(kVG, nt - m0);
            for (int g = 0; g < kVG; ++g) p.tv[g] = pl->turns32[std::min(m0 + g, nt - 1)];
            dim3 gv((W + kVCols - 1) / kVCols, nbh);
            kv<<<gv, kVCols * kVG, sm_v, s>>>(p);
            for (int g = 0; g < p.n_terms; ++g) {
                p.slot = g;
                p.a = pl->a32[m0 + g];
                p.t = pl->turns32[m0 + g];
                p.first = m0 + g == 0;
                dim3 gh((H + 63) / 64, nbw, 2);
                lr_horz<<<gh, 64, 0, s>>>(p);
            }
        }
        dim3 gf((W + 31) / 32, (H + 31) / 32);
        lr_final<<<gf, dim3(32, 8), 0, s>>>(
            p.Acc, img.out + (long long)ch * img.out_z,
            img.q_out ? img.q_out + (long long)ch * img.out_z : nullptr, H, W, p.Hp, img.out_px,
            img.q_scale);
    }
    return cudaGetLastError();
}

}  // namespace bf

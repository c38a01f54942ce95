// Forward filter for the 3-pass box at large half-widths r (support 3r > 24).
//
// A tile plus a 3r halo no longer fits on chip, so the separable filter is
// run as two streaming sweeps, the terms' filtered auxiliary images passing
// through device memory once:
//
//   lr_vert : one thread per image column and term (four terms per block,
//             sharing a ring of f; all terms in one launch while their planes
//             fit 4 GiB), walking down a band of rows (f loaded a few rows
//             ahead).  The four auxiliary images of the term (cos, sin,
//             f cos, f sin of omega f, Section 2.3) are generated on the fly
//             and filtered by the three cascaded boxes with running sums;
//             written in a blocked column layout (rows in blocks of 16, a
//             column's 16 rows contiguous) so that the second sweep reads
//             coalesced.
//   lr_horz : one thread per image row, plane and term of a launch of at most
//             eight terms, walking along a band of columns of the blocked
//             planes: the same three cascaded boxes horizontally, then the
//             per-pixel combine of eq. (final-form) into the term's own Q or P
//             accumulator slot.
//   lr_final: out = P / Q with P and Q summed over the slots, back to
//             row-major.
//
// Running sums without per-pass history.  Box k of the cascade at position q
// needs its input at q + r and q - r - 1.  Keeping one running sum per
// position that a later box needs (three for the first box, two for the
// second, one for the third, spaced L = 2r + 1 apart) makes every update read
// only the raw input at the four positions e, e - L, e - 2L, e - 3L: the
// newest is generated (or loaded); the other three come from a shared-memory
// ring of f, the planes being regenerated (lr_vert), or are read again from
// the blocked planes (lr_horz).  Each running sum is a plain sliding
// sum (add the incoming, subtract the outgoing), so rounding grows like the
// usual running sum, and the half-width r is a run-time value.  The sums start
// at zero 3r positions before the first output with the input taken as zero
// before that point, so the first 6r steps of a band are warm-up.
#include <algorithm>
#include <vector>
#include <type_traits>

#include "bf_internal.h"
#include "bf_tile.cuh"

namespace bf {

namespace {


constexpr int kVB = 4;     // lr_vert: terms per block (they share the f ring)
constexpr int kVMax = 64;  // most terms one lr_vert launch filters
constexpr int kHG = 8;     // most terms one lr_horz launch filters (accumulator slots)
#ifndef BF_LR_HWARPS
#define BF_LR_HWARPS 2048
#endif
constexpr int kHWarps = BF_LR_HWARPS;  // lr_horz: target warps per launch (sets the bands)

struct LrParams {
    const void *in;       // first pixel of the plane being filtered
    long long in_stride;  // elements between rows
    int dtype, in_px;     // element type; elements between adjacent pixels
    int H, W, r;
    int band_h, band_w;
    int n_terms;          // terms of this launch (lr_vert <= kVMax, lr_horz <= kHG)
    float tv[kVMax];      // lr_vert: turns per gray level of its terms
    float th[kHG], ah[kHG];  // lr_horz: turns and weights of its terms
    int h0;               // lr_horz: Vt slot of its first term
    int nyb;              // row blocks of the blocked column layout: ceil(H / kYB)
    float *Vt;            // [lr_vert's terms][4 planes] blocked planes: vertically filtered
    float *Acc;           // [kHG slots][2] blocked planes: Q and P per term slot
    float *ft;            // blocked plane: the channel's f
    int first;            // lr_horz: first launch of the channel (the slots start from zero)
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

// Blocked column layout of the intermediate planes: rows in blocks of kYB;
// within a block, column x holds its kYB rows contiguously and the columns
// follow each other, so pixel (x, y) sits at
//   (y / kYB) * W * kYB + x * kYB + y % kYB.
// A warp of the horizontal sweep (kYB rows of one block) then finds the
// column c of its rows at a fixed offset c * kYB from its row block: every
// step of a chunk is an immediate offset from one pointer.
constexpr int kYB = 16;

__host__ __device__ __forceinline__ size_t blocked_plane(int H, int W) {
    return (size_t)((H + kYB - 1) / kYB) * (size_t)W * kYB;
}

__device__ __forceinline__ size_t blocked_at(int W, int x, int y) {
    return (size_t)(y / kYB) * (size_t)W * kYB + (size_t)x * kYB + (y % kYB);
}

template <int DT>
__device__ __forceinline__ float load_px(const LrParams &p, int y, int x) {
    const long long off = (long long)y * p.in_stride + (long long)x * p.in_px;
    if constexpr (DT == 0) return __ldg(reinterpret_cast<const float *>(p.in) + off);
    else return (float)__ldg(reinterpret_cast<const uint8_t *>(p.in) + off);
}

constexpr int kVCols = 32;    // lr_vert: columns per block
constexpr int kChunk = 8;     // lr_vert: steps between barriers / whose loads are issued together

// The four auxiliary planes of one pixel value (cos, sin, f cos, f sin).
// The products are rounded explicitly (__fmul_rn is never fused into an
// FMA): a value regenerated from the f ring must equal, bit for bit, the one
// generated when it entered, or the running sums lose the exact shifted-copy
// relation between them and their rounding errors integrate (error growing
// like n^2.5 over an n-row band instead of n^0.5).
__device__ __forceinline__ void aux4(float tm, float fv, float (&x)[4]) {
    float r = __fmul_rn(tm, fv);
    r = r - rintf(r);
    float sn, cs;
    __sincosf(kTwoPi * r, &sn, &cs);
    x[0] = cs;
    x[1] = sn;
    x[2] = __fmul_rn(fv, cs);
    x[3] = __fmul_rn(fv, sn);
}

// The same four values as pairs: x[0] = (cos, sin), x[1] = (f cos, f sin).
__device__ __forceinline__ void aux4p(float tm, float fv, float2 (&x)[2]) {
    float r = __fmul_rn(tm, fv);
    r = r - rintf(r);
    float sn, cs;
    __sincosf(kTwoPi * r, &sn, &cs);
    x[0] = make_float2(cs, sn);
    x[1] = make_float2(__fmul_rn(fv, cs), __fmul_rn(fv, sn));
}

// grid: (ceil(W / kVCols), bands, ceil(terms / kVB)); block: kVCols x kVB
// threads, thread (column, term g) computes the four planes of term g for one
// column.  The kVB terms of a block share one ring of the last ring_size(r)
// values of f per column
// (every thread writes the same value into it; a barrier per chunk keeps the
// warps within kChunk steps of each other, far less than the ring's slack).
// Chunks are aligned so that step d of a chunk produces output row
// 8k + d of the band: the eight outputs of a chunk stay in registers and
// leave as two 16-byte stores per plane.  Dynamic smem: the f ring.
template <int DT>
__global__ void __launch_bounds__(kVCols * kVB) lr_vert(const __grid_constant__ LrParams p) {
    extern __shared__ float lv_sm[];
    const int tid = threadIdx.x;
    const int col = tid % kVCols;
    const int g = blockIdx.z * kVB + tid / kVCols;
    const int xb = blockIdx.x * kVCols;
    const int xc = min(xb + col, p.W - 1);
    const bool term_ok = g < p.n_terms;
    const float tm = p.tv[min(g, p.n_terms - 1)];
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
    const size_t plane = blocked_plane(p.H, p.W);
    float *dst = p.Vt + (size_t)g * 4 * plane;
    // running sums of the plane pairs (cos, sin) [index 0] and (f cos, f sin)
    // [index 1], one f32x2 instruction per pair and update
    float2 s1[2][3], s2[2][2], s3[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        s1[q][0] = s1[q][1] = s1[q][2] = make_float2(0.f, 0.f);
        s2[q][0] = s2[q][1] = make_float2(0.f, 0.f);
        s3[q] = make_float2(0.f, 0.f);
    }
    float cur[kChunk], nxt[kChunk];
#pragma unroll
    for (int d = 0; d < kChunk; ++d) cur[d] = load_px<DT>(p, min(max(e_s + d, 0), p.H - 1), xc);
    float2 st[2][kChunk];
    // one step; CHECKED covers steps before p0 + 3L (inputs before p0 are
    // zero) and the band's last chunk
    auto step = [&](int e, int d, auto checked) {
        constexpr bool CHECKED = decltype(checked)::value;
        const float fv = cur[d];
        ring[(e & M) * kVCols] = fv;
        float2 x0[2], x1[2], x2[2], x3[2];
        aux4p(tm, fv, x0);
        if (!CHECKED) {
            aux4p(tm, ring[((e - L) & M) * kVCols], x1);
            aux4p(tm, ring[((e - 2 * L) & M) * kVCols], x2);
            aux4p(tm, ring[((e - 3 * L) & M) * kVCols], x3);
        } else {
            const float2 z = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 2; ++q) x1[q] = x2[q] = x3[q] = z;
            if (e < p0) {
#pragma unroll
                for (int q = 0; q < 2; ++q) x0[q] = z;
            }
            if (e >= p0 + L) aux4p(tm, ring[((e - L) & M) * kVCols], x1);
            if (e >= p0 + 2 * L) aux4p(tm, ring[((e - 2 * L) & M) * kVCols], x2);
            if (e >= p0 + 3 * L) aux4p(tm, ring[((e - 3 * L) & M) * kVCols], x3);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            s1[q][0] = f2add(s1[q][0], f2sub(x0[q], x1[q]));
            s1[q][1] = f2add(s1[q][1], f2sub(x1[q], x2[q]));
            s1[q][2] = f2add(s1[q][2], f2sub(x2[q], x3[q]));
            s2[q][0] = f2add(s2[q][0], f2sub(s1[q][0], s1[q][1]));
            s2[q][1] = f2add(s2[q][1], f2sub(s1[q][1], s1[q][2]));
            s3[q] = f2add(s3[q], f2sub(s2[q][0], s2[q][1]));
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
            // tb is a multiple of 8: the chunk's rows lie in one row block
            float *dc = dst + blocked_at(p.W, xb + col, tb);
            if (tb + kChunk <= y1) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    float4 *d4 = reinterpret_cast<float4 *>(dc + 2 * q * plane);
                    d4[0] = make_float4(st[q][0].x, st[q][1].x, st[q][2].x, st[q][3].x);
                    d4[1] = make_float4(st[q][4].x, st[q][5].x, st[q][6].x, st[q][7].x);
                    d4 = reinterpret_cast<float4 *>(dc + (2 * q + 1) * plane);
                    d4[0] = make_float4(st[q][0].y, st[q][1].y, st[q][2].y, st[q][3].y);
                    d4[1] = make_float4(st[q][4].y, st[q][5].y, st[q][6].y, st[q][7].y);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 2; ++q)
#pragma unroll
                    for (int d = 0; d < kChunk; ++d)
                        if (tb + d < y1) {
                            dc[2 * q * plane + d] = st[q][d].x;
                            dc[(2 * q + 1) * plane + d] = st[q][d].y;
                        }
            }
        }
#pragma unroll
        for (int d = 0; d < kChunk; ++d) cur[d] = nxt[d];
    }
}

// f of one channel, row-major -> blocked column layout (32 x 33 shared tile).
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
        if (x < p.W && y < p.H) p.ft[blocked_at(p.W, x, y)] = tile[threadIdx.x][i];
    }
}

// grid: (ceil(nyb / 4), bands along x, 2 * terms of the group); block: 128
// threads = four warps, one row block (kYB = 16 rows) each.  blockIdx.z =
// 2 * slot + pair: pair 0 filters the (cos, sin) planes of the group's term
// `slot` into Q, pair 1 the (f cos, f sin) planes into P.  In a warp, lanes
// 0-15 carry the first plane of the pair and lanes 16-31 the second, for the
// same 16 rows; at an output the two halves meet through one shuffle.  Each
// term of the group accumulates into its own slot of Acc (summed by
// lr_final), so the group's terms run concurrently without sharing an
// accumulator.  The inputs at e - L, e - 2L, e - 3L are read again from the
// blocked planes (L2) rather than kept, so no shared memory limits the
// number of resident warps.
constexpr int kChunkG = 8;
__global__ void __launch_bounds__(128) lr_horz(const __grid_constant__ LrParams p) {
    const int lane = threadIdx.x & 31;
    const int half = lane >> 4;  // 0: cos-like plane, 1: sin-like plane
    const int pr = blockIdx.z & 1;
    const int slot = blockIdx.z >> 1;
    const int yb = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (yb >= p.nyb) return;  // whole warp
    const int y = yb * kYB + (lane & (kYB - 1));
    const int W = p.W;
    const size_t plane = blocked_plane(p.H, W);
    const size_t row = blocked_at(W, 0, min(y, p.H - 1));  // column 0 of this lane's row
    const float *V = p.Vt + ((size_t)(p.h0 + slot) * 4 + 2 * pr + half) * plane + row;
    const float *F = p.ft + row;
    float *A = p.Acc + ((size_t)slot * 2 + pr) * plane + row;
    const int x0 = blockIdx.y * p.band_w;
    const int x1 = min(x0 + p.band_w, W);
    const int r = p.r, L = 2 * r + 1;
    const int p0 = x0 - 3 * r;  // inputs before p0 count as zero
    const int e_end = x1 + 3 * r;
    const float am = p.ah[slot], tm = p.th[slot];
    // cos(x) = sin(x + quarter turn): each half evaluates one sine
    const float ph = half ? 0.f : 0.25f;
    const bool store = half == 0 && y < p.H;
    const bool first = p.first;
    float s1a = 0.f, s1b = 0.f, s1c = 0.f, s2a = 0.f, s2b = 0.f, s3 = 0.f;
    for (int e0 = p0; e0 < e_end; e0 += kChunkG) {
        // the plane at e, e - L, e - 2L, e - 3L for the chunk's steps (0 before p0)
        float cv[kChunkG][4];
        const bool edge = max(e0 - 3 * L, p0) < 0 || e0 + kChunkG > W;  // uniform
        if (!edge) {
            const float *v0 = V + (ptrdiff_t)e0 * kYB;
#pragma unroll
            for (int d = 0; d < kChunkG; ++d) cv[d][0] = __ldg(v0 + d * kYB);
#pragma unroll
            for (int k = 1; k < 4; ++k) {
                const int rel = e0 - k * L - p0;  // step d valid iff rel + d >= 0
                const float *vk = v0 - (ptrdiff_t)k * L * kYB;
                if (rel >= 0) {
#pragma unroll
                    for (int d = 0; d < kChunkG; ++d) cv[d][k] = __ldg(vk + d * kYB);
                } else if (rel > -kChunkG) {
#pragma unroll
                    for (int d = 0; d < kChunkG; ++d) {
                        const float v = __ldg(vk + max(d, -rel) * kYB);
                        cv[d][k] = rel + d >= 0 ? v : 0.f;
                    }
                } else {
#pragma unroll
                    for (int d = 0; d < kChunkG; ++d) cv[d][k] = 0.f;
                }
            }
        } else {
#pragma unroll
            for (int d = 0; d < kChunkG; ++d) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int pos = e0 + d - k * L;
                    const float v = __ldg(V + (ptrdiff_t)min(max(pos, 0), W - 1) * kYB);
                    cv[d][k] = pos >= p0 ? v : 0.f;
                }
            }
        }
        const int t0 = e0 - 3 * r;  // output column of step 0
        if (t0 + kChunkG <= x0) {
            // warm-up chunk: no outputs
#pragma unroll
            for (int d = 0; d < kChunkG; ++d) {
                s1a += cv[d][0] - cv[d][1];
                s1b += cv[d][1] - cv[d][2];
                s1c += cv[d][2] - cv[d][3];
                s2a += s1a - s1b;
                s2b += s1b - s1c;
                s3 += s2a - s2b;
            }
            continue;
        }
        // the pixel value and the slot's accumulator at the chunk's outputs
        float cf[kChunkG], ca[kChunkG];
        if (t0 >= x0 && t0 + kChunkG <= x1) {  // uniform
            const float *f0 = F + (ptrdiff_t)t0 * kYB;
            const float *a0 = A + (ptrdiff_t)t0 * kYB;
#pragma unroll
            for (int d = 0; d < kChunkG; ++d) {
                cf[d] = __ldg(f0 + d * kYB);
                ca[d] = first ? 0.f : a0[d * kYB];
            }
        } else {
#pragma unroll
            for (int d = 0; d < kChunkG; ++d) {
                const ptrdiff_t o = (ptrdiff_t)min(max(t0 + d, 0), W - 1) * kYB;
                cf[d] = __ldg(F + o);
                ca[d] = first ? 0.f : A[o];
            }
        }
        // steps past e_end (last chunk) run on clamped inputs and store nothing
        float o3[kChunkG];
#pragma unroll
        for (int d = 0; d < kChunkG; ++d) {
            s1a += cv[d][0] - cv[d][1];
            s1b += cv[d][1] - cv[d][2];
            s1c += cv[d][2] - cv[d][3];
            s2a += s1a - s1b;
            s2b += s1b - s1c;
            s3 += s2a - s2b;
            o3[d] = s3;
        }
#pragma unroll
        for (int d = 0; d < kChunkG; ++d) {
            float rr = fmaf(tm, cf[d], ph);
            rr = rr - rintf(rr);
            const float mine = am * __sinf(kTwoPi * rr) * o3[d];
            const float other = __shfl_down_sync(0xffffffffu, mine, 16);
            const int t = t0 + d;
            if (store && t >= x0 && t < x1) A[(ptrdiff_t)t * kYB] = ca[d] + (mine + other);
        }
    }
}

// out = P / Q, with Q and P the sums over the used term slots of Acc (in
// slot order), blocked column layout -> row-major through a 32 x 33 shared
// tile.
// grid: (ceil(W / 32), ceil(H / 32)); block: (32, 8)
__global__ void lr_final(const float *__restrict__ Acc, int n_slots, float *__restrict__ out,
                         float *__restrict__ q_out, int H, int W, int out_px, float q_scale) {
    __shared__ float tp[32][33];
    __shared__ float tq[32][33];
    const size_t plane = blocked_plane(H, W);
    const int xb = blockIdx.x * 32, yb = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int x = xb + i, y = yb + threadIdx.x;
        if (x < W && y < H) {
            const size_t o = blocked_at(W, x, y);
            float q = Acc[o], pp = Acc[plane + o];
            for (int s = 1; s < n_slots; ++s) {
                q += Acc[2 * s * plane + o];
                pp += Acc[(2 * s + 1) * plane + o];
            }
            tq[i][threadIdx.x] = q;
            tp[i][threadIdx.x] = pp;
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

// Terms per lr_vert launch: all of them while their filtered planes stay
// within 4 GiB, else fewer (at least one lr_horz launch's worth).
static int vert_terms(const bf_plan *pl, int H, int W) {
    const size_t term_bytes = 4 * blocked_plane(H, W) * sizeof(float);
    const size_t budget = (size_t)4 << 30;
    const int nt = (int)pl->a32.size();
    const int cap = (int)std::max<size_t>(kHG, std::min<size_t>(kVMax, budget / term_bytes));
    return std::min(nt, cap);
}

size_t large_workspace(const bf_plan *pl, int H, int W) {
    const size_t planes = 4 * (size_t)vert_terms(pl, H, W) + 2 * kHG + 1;
    return planes * blocked_plane(H, W) * sizeof(float) + 256;
}

cudaError_t launch_large_box(const bf_plan *pl, const BfImage &img, void *ws, cudaStream_t s) {
    const int H = img.H, W = img.W;
    const int nt = (int)pl->a32.size();
    char *base = reinterpret_cast<char *>(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    LrParams p{};
    p.in_stride = img.in_row_stride;
    p.dtype = img.dtype;
    p.in_px = img.in_px;
    p.H = H;
    p.W = W;
    p.nyb = (H + kYB - 1) / kYB;
    p.r = pl->r_box;
    const int gv_max = vert_terms(pl, H, W);
    const size_t plane = blocked_plane(H, W);
    p.Vt = reinterpret_cast<float *>(base);
    p.Acc = p.Vt + (size_t)4 * gv_max * plane;
    p.ft = p.Acc + (size_t)2 * kHG * plane;
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
    int n_sm = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kv, kVCols * kVB, sm_v);
    if (e != cudaSuccess) return e;
    const int resident_vert = std::max(1, n_sm * per_sm);

    // lr_horz launches: ceil(nt / kHG) of them, sizes as equal as possible
    // and non-increasing (the first launch, which starts every slot from
    // zero, is the largest); each lr_vert launch covers whole lr_horz launches.
    const int n_h = (nt + kHG - 1) / kHG;
    std::vector<int> h_size(n_h);
    for (int i = 0; i < n_h; ++i) h_size[i] = nt / n_h + (i < nt % n_h ? 1 : 0);

    // Bands.  lr_vert's (multiples of 8 rows): as many as one wave of
    // resident blocks holds (a partial second wave costs a whole band's time).
    // lr_horz's: about 2048 warps in all, which keeps the working set of the
    // trailing reads in L2.  Both stay at least 12r long (the 6r warm-up at
    // most half a band).
    const int min_band = 12 * p.r;
    const int ncb = (W + kVCols - 1) / kVCols;
    const int zb_max = (gv_max + kVB - 1) / kVB;
    const int nbh_max = std::max(1, std::min(resident_vert / (ncb * zb_max), H / min_band));
    p.band_h = ((H + nbh_max - 1) / nbh_max + 7) / 8 * 8;
    const int nbh = (H + p.band_h - 1) / p.band_h;
    const int g_warps = p.nyb * 2 * h_size[0];
    const int nbw_max = std::max(1, std::min((kHWarps + g_warps / 2) / g_warps, W / min_band));
    p.band_w = ((W + nbw_max - 1) / nbw_max + 7) / 8 * 8;
    const int nbw = (W + p.band_w - 1) / p.band_w;

    const int esz = img.dtype == 0 ? 4 : 1;
    for (int ch = 0; ch < img.C; ++ch) {
        p.in = reinterpret_cast<const char *>(img.in) + (long long)ch * img.in_z * esz;
        dim3 gt((W + 31) / 32, (H + 31) / 32);
        kt<<<gt, dim3(32, 8), 0, s>>>(p);
        int h = 0, m0 = 0;
        while (h < n_h) {
            // lr_horz launches [h, h1) fit one lr_vert launch
            int h1 = h, nv = 0;
            while (h1 < n_h && nv + h_size[h1] <= gv_max) nv += h_size[h1++];
            if (h1 == h) return cudaErrorInvalidValue;  // cannot happen: h_size <= kHG <= gv_max
            p.n_terms = nv;
            for (int g = 0; g < kVMax; ++g) p.tv[g] = pl->turns32[m0 + std::min(g, nv - 1)];
            dim3 gv(ncb, nbh, (nv + kVB - 1) / kVB);
            kv<<<gv, kVCols * kVB, sm_v, s>>>(p);
            int off = 0;
            for (; h < h1; ++h) {
                p.n_terms = h_size[h];
                p.h0 = off;
                for (int g = 0; g < kHG; ++g) {
                    const int m = m0 + off + std::min(g, h_size[h] - 1);
                    p.th[g] = pl->turns32[m];
                    p.ah[g] = pl->a32[m];
                }
                p.first = h == 0;
                dim3 gh((p.nyb + 3) / 4, nbw, 2 * p.n_terms);
                lr_horz<<<gh, 128, 0, s>>>(p);
                off += h_size[h];
            }
            m0 += nv;
        }
        dim3 gf((W + 31) / 32, (H + 31) / 32);
        lr_final<<<gf, dim3(32, 8), 0, s>>>(
            p.Acc, h_size[0], img.out + (long long)ch * img.out_z,
            img.q_out ? img.q_out + (long long)ch * img.out_z : nullptr, H, W, img.out_px,
            img.q_scale);
    }
    return cudaGetLastError();
}

}  // namespace bf

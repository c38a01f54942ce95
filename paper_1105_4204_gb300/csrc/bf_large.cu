// Streaming forward filters: the 3-pass box at large half-widths r (support
// 3r > 24) and, further down, the recursive Gaussian (rg_*), which share the
// blocked layout, the transpose, the horizontal warp layout with its on-chip
// term reduction, and the final division.
//
// Large box.  A tile plus a 3r halo no longer fits on chip, so the separable
// filter is run as two streaming sweeps, the terms' filtered auxiliary images
// passing through device memory once:
//
//   lr_vert : one thread per image column and term (four terms per block,
//             sharing a ring of f; all terms in one launch while their planes
//             fit 4 GiB), walking down a band of rows (f loaded a few rows
//             ahead).  The four auxiliary images of the term (cos, sin,
//             f cos, f sin of omega f, Section 2.3) are generated on the fly
//             and filtered by the three cascaded boxes with running sums, as
//             two pairs (cos, sin) and (f cos, f sin); written pair-
//             interleaved in a blocked column layout (rows in blocks of 16, a
//             column's 16 rows contiguous) so that the second sweep reads
//             coalesced.
//   lr_horz : one warp per term, pair and two row blocks (a lane per row,
//             the pair as a float2), the warps of four terms in one block
//             walking along a band of columns in step: the same three
//             cascaded boxes horizontally, the per-pixel combine of
//             eq. (final-form), and the block's four terms summed on chip into
//             one Q and one P slot per group, written once.
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
constexpr int kHT = 4;     // lr_horz: terms per block (summed on chip into one slot)
constexpr int kVMax = 64;  // most terms one lr_vert launch filters
// lr_horz: L2 bytes the lagged reads of all resident blocks may occupy
constexpr size_t kHorzL2Bytes = (size_t)56 << 20;
constexpr int kHorzPrefetchR = 24;  // lr_horz prefetches the next chunk from this r on
__host__ __device__ __forceinline__ int L_of(int r) { return 2 * r + 1; }

struct LrParams {
    const void *in;       // first pixel of the plane being filtered
    long long in_stride;  // elements between rows
    int dtype, in_px;     // element type; elements between adjacent pixels
    int H, W, r;
    int band_h, band_w;
    int n_terms;          // terms of this launch (<= kVMax; lr_horz takes lr_vert's)
    float tv[kVMax];      // lr_vert: turns per gray level of its terms
    float th[kVMax], ah[kVMax];  // lr_horz: turns and weights of its terms
    int nyb;              // row blocks of the blocked column layout: ceil(H / kYB)
    float *Vt;            // [lr_vert's terms][4 planes] blocked planes: vertically filtered
    float *Acc;           // [slots][2] blocked planes: Q and P per group of kHT terms
    float *ft;            // blocked plane: the channel's f
    int first;            // lr_horz: first launch of the channel (the slots start from zero)
};

// lr_vert / rg_vert: steps between barriers / whose loads are issued together
// (a divisor of the 16-row blocks; 16 measured slower: fewer resident blocks)
constexpr int kChunk = 8;
static_assert(16 % kChunk == 0, "chunks must not straddle row blocks");

// Power-of-two size of lr_vert's shared f ring (which has kChunk more slots
// mirroring its first kChunk): the 3L + 1 values a stream needs, plus slack for the warps sharing it to be up to two chunks apart
// (they meet at a barrier every chunk) without overwriting a value another
// warp still has to read.
__host__ __device__ __forceinline__ int ring_size(int r) {
    int n = 1;
    while (n < 3 * (2 * r + 1) + 1 + 2 * kChunk) n <<= 1;
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

// The four auxiliary planes of one pixel value (cos, sin, f cos, f sin).
// The products are rounded explicitly (__fmul_rn is never fused into an
// FMA): a value regenerated from the f ring must equal, bit for bit, the one
// generated when it entered, or the running sums lose the exact shifted-copy
// relation between them and their rounding errors integrate (error growing
// like n^2.5 over an n-row band instead of n^0.5).
// As pairs: x[0] = (cos, sin), x[1] = (f cos, f sin).
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
    // pair q of term g: float2 blocked plane at Vt + (2 g + q) * 2 * plane
    float2 *dst = reinterpret_cast<float2 *>(p.Vt) + (size_t)g * 2 * plane;
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
    // r1, r2, r3: ring slots of e0 - L, e0 - 2L, e0 - 3L for the chunk at e0;
    // a chunk's window never wraps (the first kChunk slots are mirrored past
    // the end of the ring), so step d reads at a fixed offset d * kVCols.
    const float *r1 = ring, *r2 = ring, *r3 = ring;
    auto step = [&](int e, int d, auto checked) {
        constexpr bool CHECKED = decltype(checked)::value;
        const float fv = cur[d];
        const int slot = e & M;
        ring[slot * kVCols] = fv;
        if (slot < kChunk) ring[(slot + RS) * kVCols] = fv;
        float2 x0[2], x1[2], x2[2], x3[2];
        aux4p(tm, fv, x0);
        if (!CHECKED) {
            aux4p(tm, r1[d * kVCols], x1);
            aux4p(tm, r2[d * kVCols], x2);
            aux4p(tm, r3[d * kVCols], x3);
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
        const int tb = e0 - 3 * r;  // output row of step d = 0 (tb - y0 is a multiple of kChunk)
        const bool fast = e0 >= p0 + 3 * L && e0 + kChunk <= e_end;  // uniform
        if (fast) {
            r1 = ring + ((e0 - L) & M) * kVCols;
            r2 = ring + ((e0 - 2 * L) & M) * kVCols;
            r3 = ring + ((e0 - 3 * L) & M) * kVCols;
#pragma unroll
            for (int d = 0; d < kChunk; ++d) step(e0 + d, d, std::false_type{});
        } else {
#pragma unroll
            for (int d = 0; d < kChunk; ++d)
                if (e0 + d < e_end) step(e0 + d, d, std::true_type{});
        }
        if (col_ok && tb >= y0) {
            // tb is a multiple of kChunk: the chunk's rows lie in one row block
            float2 *dc = dst + blocked_at(p.W, xb + col, tb);
            if (tb + kChunk <= y1) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    float4 *d4 = reinterpret_cast<float4 *>(dc + q * plane);
#pragma unroll
                    for (int k = 0; k < kChunk / 2; ++k)
                        d4[k] = make_float4(st[q][2 * k].x, st[q][2 * k].y, st[q][2 * k + 1].x,
                                            st[q][2 * k + 1].y);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 2; ++q)
#pragma unroll
                    for (int d = 0; d < kChunk; ++d)
                        if (tb + d < y1) dc[q * plane + d] = st[q][d];
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

// Persistent: block b takes work items b, b + gridDim.x, ... where an item is
// (two row blocks, a band of columns, a group of kHT terms); the grid is
// sized so that the lagged reads of all resident blocks stay in L2 (each
// lane reads back the 3L columns behind it).  Block: 2 kHT warps.  Warp w
// takes term w / 2 of the item's group and pair w % 2 (0: the (cos, sin)
// planes, whose combine goes to Q; 1: (f cos, f sin), to P); lane l carries
// row l % 16 of the item's row block l / 16, both planes of the pair in one
// float2.  All warps of a block walk the same columns in step, kChunkH at a
// time, the loads of the next chunk issued before the current one is
// filtered.  Per chunk every warp turns its filtered pair into the term's
// contribution a_m (cos(w f) W[.cos] + sin(w f) W[.sin]) at the chunk's
// outputs; the block sums the contributions of its terms in term order
// through shared memory and writes the group's Q and P slot once (adding to
// it when the terms of the image did not fit one lr_vert launch).  lr_final
// sums the slots in slot order.
//
// PF (large r): the next chunk's loads are issued before the current chunk is
// filtered (two register buffers, one block per SM).  Without PF (smaller r,
// whose lagged reads are closer and more likely in L2) a chunk's loads are
// issued when it starts, and two blocks fit an SM.
constexpr int kChunkH = 8;
template <bool PF>
__global__ void __launch_bounds__(64 * kHT, PF ? 1 : 2) lr_horz(const __grid_constant__ LrParams p) {
    __shared__ float hs_sm[2][2 * kHT][kChunkH][32];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int q = warp & 1;
    const int tl = warp >> 1;
    const int W = p.W;
    const size_t plane = blocked_plane(p.H, W);
    const int r = p.r, L = 2 * r + 1;
    const float2 z2 = make_float2(0.f, 0.f);
    // reduction role: thread -> (pair rq, step rd, lane rl) outputs of a chunk
    constexpr int NOUT = 2 * kChunkH * 32;
    constexpr int PER = NOUT / (64 * kHT);
    static_assert(NOUT % (64 * kHT) == 0, "reduction split");
    const int nyb2 = (p.nyb + 1) / 2;
    const int nbw = (W + p.band_w - 1) / p.band_w;
    const int n_groups = (p.n_terms + kHT - 1) / kHT;
    const int n_items = nyb2 * nbw * n_groups;
    int buf = 0;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int iy = item % nyb2;
        const int ix = (item / nyb2) % nbw;
        const int gz = item / (nyb2 * nbw);
        const int term = gz * kHT + tl;
        const bool term_ok = term < p.n_terms;  // uniform per warp
        const int tc = min(term, p.n_terms - 1);
        const int rb = min(iy * 2 + (lane >> 4), p.nyb - 1);
        const int y_lane = rb * kYB + (lane & (kYB - 1));
        const size_t row = blocked_at(W, 0, min(y_lane, p.H - 1));  // column 0 of this row
        const float2 *V =
            reinterpret_cast<const float2 *>(p.Vt) + ((size_t)tc * 2 + q) * plane + row;
        const float *F = p.ft + row;
        const int x0 = ix * p.band_w;
        const int x1 = min(x0 + p.band_w, W);
        const int p0 = x0 - 3 * r;  // inputs before p0 count as zero
        const int e_end = x1 + 3 * r;
        const float am = term_ok ? p.ah[tc] : 0.f, tm = p.th[tc];
        float2 s1a = z2, s1b = z2, s1c = z2, s2a = z2, s2b = z2, s3 = z2;
        // the pair at e, e - L, e - 2L, e - 3L for the steps of the chunk at e0
        // (0 before p0), and the pixel value at its outputs
        auto load = [&](int e0, float2 (&cv)[kChunkH][4], float (&cf)[kChunkH]) {
            const bool edge = max(e0 - 3 * L, p0) < 0 || e0 + kChunkH > W;  // uniform
            if (!edge) {
                const float2 *v0 = V + (ptrdiff_t)e0 * kYB;
#pragma unroll
                for (int d = 0; d < kChunkH; ++d) cv[d][0] = __ldg(v0 + d * kYB);
#pragma unroll
                for (int k = 1; k < 4; ++k) {
                    const int rel = e0 - k * L - p0;  // step d valid iff rel + d >= 0
                    const float2 *vk = v0 - (ptrdiff_t)k * L * kYB;
                    if (rel >= 0) {
#pragma unroll
                        for (int d = 0; d < kChunkH; ++d) cv[d][k] = __ldg(vk + d * kYB);
                    } else if (rel > -kChunkH) {
#pragma unroll
                        for (int d = 0; d < kChunkH; ++d) {
                            const float2 v = __ldg(vk + max(d, -rel) * kYB);
                            cv[d][k] = rel + d >= 0 ? v : z2;
                        }
                    } else {
#pragma unroll
                        for (int d = 0; d < kChunkH; ++d) cv[d][k] = z2;
                    }
                }
            } else {
#pragma unroll
                for (int d = 0; d < kChunkH; ++d) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int pos = e0 + d - k * L;
                        const float2 v = __ldg(V + (ptrdiff_t)min(max(pos, 0), W - 1) * kYB);
                        cv[d][k] = pos >= p0 ? v : z2;
                    }
                }
            }
            const int t0 = e0 - 3 * r;
            if (t0 >= x0 && t0 + kChunkH <= x1) {  // uniform
                const float *f0 = F + (ptrdiff_t)t0 * kYB;
#pragma unroll
                for (int d = 0; d < kChunkH; ++d) cf[d] = __ldg(f0 + d * kYB);
            } else {
#pragma unroll
                for (int d = 0; d < kChunkH; ++d)
                    cf[d] = __ldg(F + (ptrdiff_t)min(max(t0 + d, 0), W - 1) * kYB);
            }
        };
        // one chunk: prefetch the next one into (nxt, nxtf), filter (cur, curf)
        auto body = [&](int e0, float2 (&cur)[kChunkH][4], float (&curf)[kChunkH],
                        float2 (&nxt)[kChunkH][4], float (&nxtf)[kChunkH]) {
            if constexpr (PF) {
                if (e0 + kChunkH < e_end) load(e0 + kChunkH, nxt, nxtf);
            } else {
                load(e0, cur, curf);
            }
            const int t0 = e0 - 3 * r;  // output column of step 0
            if (t0 + kChunkH <= x0) {
                // warm-up chunk: no outputs (uniform over the block)
#pragma unroll
                for (int d = 0; d < kChunkH; ++d) {
                    s1a = f2add(s1a, f2sub(cur[d][0], cur[d][1]));
                    s1b = f2add(s1b, f2sub(cur[d][1], cur[d][2]));
                    s1c = f2add(s1c, f2sub(cur[d][2], cur[d][3]));
                    s2a = f2add(s2a, f2sub(s1a, s1b));
                    s2b = f2add(s2b, f2sub(s1b, s1c));
                    s3 = f2add(s3, f2sub(s2a, s2b));
                }
                return;
            }
            // steps past e_end (last chunk) run on clamped inputs and store nothing
#pragma unroll
            for (int d = 0; d < kChunkH; ++d) {
                s1a = f2add(s1a, f2sub(cur[d][0], cur[d][1]));
                s1b = f2add(s1b, f2sub(cur[d][1], cur[d][2]));
                s1c = f2add(s1c, f2sub(cur[d][2], cur[d][3]));
                s2a = f2add(s2a, f2sub(s1a, s1b));
                s2b = f2add(s2b, f2sub(s1b, s1c));
                s3 = f2add(s3, f2sub(s2a, s2b));
                float rr = tm * curf[d];
                rr = rr - rintf(rr);
                float sn, cs;
                __sincosf(kTwoPi * rr, &sn, &cs);
                hs_sm[buf][warp][d][lane] = am * fmaf(cs, s3.x, sn * s3.y);
            }
            __syncthreads();
            // sum the group's terms in term order and write the slot
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int o = k * 64 * kHT + threadIdx.x;
                const int rq = o / (kChunkH * 32);
                const int rd = (o / 32) % kChunkH;
                const int rl = o % 32;
                float v = hs_sm[buf][rq][rd][rl];
#pragma unroll
                for (int t = 1; t < kHT; ++t) v += hs_sm[buf][2 * t + rq][rd][rl];
                const int tcol = t0 + rd;
                const int orb = iy * 2 + (rl >> 4);
                const int oy = orb * kYB + (rl & (kYB - 1));
                if (tcol >= x0 && tcol < x1 && orb < p.nyb && oy < p.H) {
                    float *A = p.Acc + ((size_t)gz * 2 + rq) * plane + blocked_at(W, tcol, oy);
                    *A = p.first ? v : *A + v;
                }
            }
            buf ^= 1;
        };
        float2 ca[kChunkH][4], cb[kChunkH][4];
        float fa[kChunkH], fb[kChunkH];
        if constexpr (PF) {
            load(p0, ca, fa);
            // two chunks per iteration so that the buffers swap roles without copies
            for (int e0 = p0; e0 < e_end; e0 += 2 * kChunkH) {
                body(e0, ca, fa, cb, fb);
                if (e0 + kChunkH < e_end) body(e0 + kChunkH, cb, fb, ca, fa);
            }
        } else {
            for (int e0 = p0; e0 < e_end; e0 += kChunkH) body(e0, ca, fa, cb, fb);
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
            // unrolled so that the slots' loads are in flight together (the
            // sums still run in slot order)
#pragma unroll 8
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


// ---------------------------------------------------------------------------
// Recursive Gaussian (the O(1) spatial filter of the paper's experiments,
// Section 3): per axis a causal and an anticausal third-order recursion
// (Young and van Vliet), B and a_k = b_k / b0:
//   w(e) = B x(e) + a1 w(e-1) + a2 w(e-2) + a3 w(e-3)       (causal)
//   y(e) = B w(e) + a1 y(e+1) + a2 y(e+2) + a3 y(e+3)       (anticausal)
// evaluated in difference form: with d1 = w(e-1) - w(e-2), d2 = w(e-2) - w(e-3),
//   w(e) = w(e-1) + [B (x(e) - w(e-1)) - ((a2 + a3) d1 + a3 d2)],
// the same recursion (B = 1 - a1 - a2 - a3), but with unit DC gain exactly
// whatever the FP32 rounding of its coefficients, and without the
// cancellation of the direct form's large alternating terms (at sigma = 100,
// a1 ~ 3: the direct form in FP32 is off by units of gray level, this form by
// about 1e-3).  The causal pass starts from its steady state for x(0) (exact
// for the clamped extension) and runs P samples past the last one on the
// constant extension; the anticausal pass starts there from its steady state.
// The vertical pass (rg_vert, a thread per column and term, four terms per
// block) writes the filtered pairs (cos, sin) and (f cos, f sin) of every
// term through the scratch (rows 0 .. H+P-1 of an extended blocked layout);
// the horizontal pass (rg_horz, the lr_horz warp layout: a warp per term,
// pair and two row blocks, four terms per block) filters them in place along
// the rows (columns 0 .. W+P-1) and, on its way back, combines
// eq. (final-form) per pixel and sums the block's four terms on chip into one
// (Q, P) slot pair per group.

struct RgParams {
    const void *in;       // first pixel of the plane being filtered
    long long in_stride;  // elements between rows
    int dtype, in_px;
    int H, W, P;
    int We;               // columns of the extended planes, W + P rounded up to 8
    int nybe;             // row blocks of the extended planes, ceil((H + P) / 16)
    int nyb;              // row blocks of the image
    int n_terms;
    float tv[kVMax], ah[kVMax];  // turns per gray level and weights of the launch's terms
    float cB, cD1, cD2;   // B, a2 + a3, a3 of the difference form
    float *Vt;            // [terms][2 pairs] float2 planes of nybe * 16 * We
    float *Acc;           // [slots][Q, P] blocked H x W planes
    const float *ft;      // f, blocked H x W
    int first;            // first launch of the plane (slots start from zero)
};

// One step of the difference form on a pair: state (w = last output,
// d1, d2 = its last two increments).
__device__ __forceinline__ float2 rg_step1(float2 cB, float2 cD1, float2 cD2, float2 x,
                                           float2 &w, float2 &d1, float2 &d2) {
    const float2 dw = f2sub(f2mul(cB, f2sub(x, w)), f2fma(cD2, d2, f2mul(cD1, d1)));
    w = f2add(w, dw);
    d2 = d1;
    d1 = dw;
    return w;
}

__device__ __forceinline__ void rg_step(const RgParams &p, const float2 (&x)[2], float2 (&w)[2],
                                        float2 (&d1)[2], float2 (&d2)[2]) {
    const float2 cB = make_float2(p.cB, p.cB), cD1 = make_float2(p.cD1, p.cD1);
    const float2 cD2 = make_float2(p.cD2, p.cD2);
#pragma unroll
    for (int q = 0; q < 2; ++q) rg_step1(cB, cD1, cD2, x[q], w[q], d1[q], d2[q]);
}

// grid: (ceil(W / 32), 1, ceil(terms / 4)); block 128: (column, term)
template <int DT>
__global__ void __launch_bounds__(kVCols * kVB) rg_vert(const __grid_constant__ RgParams p) {
    const int tid = threadIdx.x;
    const int col = tid % kVCols;
    const int g = blockIdx.z * kVB + tid / kVCols;
    const int x = blockIdx.x * kVCols + col;
    const int xc = min(x, p.W - 1);
    const bool col_ok = x < p.W && g < p.n_terms;
    const float tm = p.tv[min(g, p.n_terms - 1)];
    const int E = p.H + p.P;
    const size_t plane = (size_t)p.nybe * kYB * p.We;
    float2 *dst = reinterpret_cast<float2 *>(p.Vt) + (size_t)min(g, p.n_terms - 1) * 2 * plane;
    auto fval = [&](int e) {
        const long long off = (long long)min(e, p.H - 1) * p.in_stride + (long long)xc * p.in_px;
        if constexpr (DT == 0) return __ldg(reinterpret_cast<const float *>(p.in) + off);
        else return (float)__ldg(reinterpret_cast<const uint8_t *>(p.in) + off);
    };
    // state: last output (steady state x(0)) and its last two increments
    float2 s1[2], s2[2], s3[2], x0[2];
    aux4p(tm, fval(0), x0);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        s1[q] = x0[q];
        s2[q] = s3[q] = make_float2(0.f, 0.f);
    }
    // f of the chunk being filtered and of the next two (loads issued two
    // chunks ahead: with few terms the sweep has few warps to hide latency)
    float cur[kChunk], nxt[kChunk], nx2[kChunk];
#pragma unroll
    for (int d = 0; d < kChunk; ++d) {
        cur[d] = fval(d);
        nxt[d] = fval(kChunk + d);
    }
    float2 st[2][kChunk];
    // causal, rows 0 .. E-1 (the last chunk's rows past E keep the state)
    for (int e0 = 0; e0 < E; e0 += kChunk) {
#pragma unroll
        for (int d = 0; d < kChunk; ++d) nx2[d] = fval(e0 + 2 * kChunk + d);
#pragma unroll
        for (int d = 0; d < kChunk; ++d) {
            if (e0 + d < E) {
                float2 xi[2];
                aux4p(tm, cur[d], xi);
                rg_step(p, xi, s1, s2, s3);
            }
            st[0][d] = s1[0];
            st[1][d] = s1[1];
        }
        if (col_ok) {
            float2 *dc = dst + blocked_at(p.We, x, e0);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float4 *d4 = reinterpret_cast<float4 *>(dc + q * plane);
#pragma unroll
                for (int k = 0; k < kChunk / 2; ++k)
                    d4[k] = make_float4(st[q][2 * k].x, st[q][2 * k].y, st[q][2 * k + 1].x,
                                        st[q][2 * k + 1].y);
            }
        }
#pragma unroll
        for (int d = 0; d < kChunk; ++d) {
            cur[d] = nxt[d];
            nxt[d] = nx2[d];
        }
    }
    // anticausal, rows E-1 .. 0, from the steady state of w(E-1), in place
    float2 t1[2], t2[2], t3[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        t1[q] = s1[q];
        t2[q] = t3[q] = make_float2(0.f, 0.f);
    }
    if (!col_ok) return;
    // the chunk at e0 of both pairs (rows e0 .. e0+7 are contiguous)
    auto load_chunk = [&](int e0, float2 (&wv)[2][kChunk]) {
        const float2 *dc = dst + blocked_at(p.We, x, e0);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float4 *s4 = reinterpret_cast<const float4 *>(dc + q * plane);
#pragma unroll
            for (int k = 0; k < kChunk / 2; ++k) {
                const float4 v = s4[k];
                wv[q][2 * k] = make_float2(v.x, v.y);
                wv[q][2 * k + 1] = make_float2(v.z, v.w);
            }
        }
    };
    float2 wv[2][kChunk], nv[2][kChunk], nv2[2][kChunk];
    const int e_top = (E - 1) / kChunk * kChunk;
    load_chunk(e_top, wv);
    if (e_top >= kChunk) load_chunk(e_top - kChunk, nv);
    for (int e0 = e_top; e0 >= 0; e0 -= kChunk) {
        // the chunk after next, issued ahead; it is read before this chunk's
        // results are written, and lies in other rows
        if (e0 >= 2 * kChunk) load_chunk(e0 - 2 * kChunk, nv2);
#pragma unroll
        for (int d = kChunk - 1; d >= 0; --d) {
            if (e0 + d < E) {
                float2 wi[2] = {wv[0][d], wv[1][d]};
                rg_step(p, wi, t1, t2, t3);
                wv[0][d] = t1[0];
                wv[1][d] = t1[1];
            }
        }
        float2 *dc = dst + blocked_at(p.We, x, e0);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            float4 *d4 = reinterpret_cast<float4 *>(dc + q * plane);
#pragma unroll
            for (int k = 0; k < kChunk / 2; ++k)
                d4[k] = make_float4(wv[q][2 * k].x, wv[q][2 * k].y, wv[q][2 * k + 1].x,
                                    wv[q][2 * k + 1].y);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int d = 0; d < kChunk; ++d) {
                wv[q][d] = nv[q][d];
                nv[q][d] = nv2[q][d];
            }
    }
}

// grid: (ceil(nyb / 2), 1, ceil(terms / kHT)); block: 2 kHT warps, as lr_horz
__global__ void __launch_bounds__(64 * kHT) rg_horz(const __grid_constant__ RgParams p) {
    __shared__ float hs_sm[2][2 * kHT][kChunkH][32];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int q = warp & 1;
    const int tl = warp >> 1;
    const int term = blockIdx.z * kHT + tl;
    const bool term_ok = term < p.n_terms;
    const int tc = min(term, p.n_terms - 1);
    const int W = p.W;
    const size_t plane = (size_t)p.nybe * kYB * p.We;
    const size_t fplane = blocked_plane(p.H, W);
    const int rb = min((int)blockIdx.x * 2 + (lane >> 4), p.nyb - 1);
    const int y_own = (int)blockIdx.x * 2 * kYB + lane;  // the lane's row (may be past H)
    const int y_lane = min(rb * kYB + (lane & (kYB - 1)), p.H - 1);
    // lanes past the last row read the last row's data and store nothing
    const bool row_ok = y_own < p.H;
    float2 *V = reinterpret_cast<float2 *>(p.Vt) + ((size_t)tc * 2 + q) * plane +
                blocked_at(p.We, 0, y_lane);
    const float *F = p.ft + blocked_at(W, 0, y_lane);
    const float am = term_ok ? p.ah[tc] : 0.f, tm = p.tv[tc];
    const int E = W + p.P;
    constexpr int NOUT = 2 * kChunkH * 32;
    constexpr int PER = NOUT / (64 * kHT);
    // causal, columns 0 .. E-1, in place (inputs past W-1 are the last one)
    float2 s1 = V[0], s2 = make_float2(0.f, 0.f), s3 = s2;
    const float2 last = V[(size_t)(W - 1) * kYB];
    const float2 cB = make_float2(p.cB, p.cB), cD1 = make_float2(p.cD1, p.cD1);
    const float2 cD2 = make_float2(p.cD2, p.cD2);
    // the chunk being filtered and the next two (loads issued two chunks
    // ahead; columns ahead of the in-place writes)
    float2 cur[kChunkH], nxt[kChunkH], nx2[kChunkH];
#pragma unroll
    for (int d = 0; d < kChunkH; ++d) {
        cur[d] = d < W ? V[(size_t)d * kYB] : last;
        nxt[d] = kChunkH + d < W ? V[(size_t)(kChunkH + d) * kYB] : last;
    }
    for (int e0 = 0; e0 < E; e0 += kChunkH) {
#pragma unroll
        for (int d = 0; d < kChunkH; ++d) {
            const int e = e0 + 2 * kChunkH + d;
            nx2[d] = e < W ? V[(size_t)e * kYB] : last;
        }
#pragma unroll
        for (int d = 0; d < kChunkH; ++d) {
            if (e0 + d < E) {
                const float2 v = rg_step1(cB, cD1, cD2, cur[d], s1, s2, s3);
                if (row_ok) V[(size_t)(e0 + d) * kYB] = v;
            }
        }
#pragma unroll
        for (int d = 0; d < kChunkH; ++d) {
            cur[d] = nxt[d];
            nxt[d] = nx2[d];
        }
    }
    // anticausal, columns E-1 .. 0, combining at the image's columns
    float2 t1 = s1, t2 = make_float2(0.f, 0.f), t3 = t2;
    int buf = 0;
    auto load_back = [&](int e0, float2 (&wv)[kChunkH], float (&cf)[kChunkH]) {
#pragma unroll
        for (int d = 0; d < kChunkH; ++d) {
            const int e = e0 + d;
            wv[d] = e < E ? V[(size_t)e * kYB] : make_float2(0.f, 0.f);
            cf[d] = __ldg(F + (size_t)min(e, W - 1) * kYB);
        }
    };
    float2 wv[kChunkH], nwv[kChunkH], nw2[kChunkH];
    float cf[kChunkH], ncf[kChunkH], nc2[kChunkH];
    const int e_top = (E - 1) / kChunkH * kChunkH;
    load_back(e_top, wv, cf);
    if (e_top >= kChunkH) load_back(e_top - kChunkH, nwv, ncf);
    // the chunk being filtered and the next two (loads issued two chunks ahead)
    auto advance = [&]() {
#pragma unroll
        for (int d = 0; d < kChunkH; ++d) {
            wv[d] = nwv[d];
            cf[d] = ncf[d];
            nwv[d] = nw2[d];
            ncf[d] = nc2[d];
        }
    };
    for (int e0 = e_top; e0 >= 0; e0 -= kChunkH) {
        if (e0 >= 2 * kChunkH) load_back(e0 - 2 * kChunkH, nw2, nc2);
#pragma unroll
        for (int d = kChunkH - 1; d >= 0; --d) {
            if (e0 + d < E) wv[d] = rg_step1(cB, cD1, cD2, wv[d], t1, t2, t3);
        }
        if (e0 >= W) {  // extension only: no outputs (uniform)
            advance();
            continue;
        }
#pragma unroll
        for (int d = 0; d < kChunkH; ++d) {
            float rr = tm * cf[d];
            rr = rr - rintf(rr);
            float sn, cs;
            __sincosf(kTwoPi * rr, &sn, &cs);
            hs_sm[buf][warp][d][lane] = am * fmaf(cs, wv[d].x, sn * wv[d].y);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int o = k * 64 * kHT + threadIdx.x;
            const int rq = o / (kChunkH * 32);
            const int rd = (o / 32) % kChunkH;
            const int rl = o % 32;
            float v = hs_sm[buf][rq][rd][rl];
#pragma unroll
            for (int t = 1; t < kHT; ++t) v += hs_sm[buf][2 * t + rq][rd][rl];
            const int tcol = e0 + rd;
            const int orb = blockIdx.x * 2 + (rl >> 4);
            const int oy = orb * kYB + (rl & (kYB - 1));
            if (tcol < W && orb < p.nyb && oy < p.H) {
                float *A = p.Acc + ((size_t)blockIdx.z * 2 + rq) * fplane + blocked_at(W, tcol, oy);
                *A = p.first ? v : *A + v;
            }
        }
        buf ^= 1;
        advance();
    }
}

}  // namespace

// Terms per lr_vert launch: all of them while their filtered planes stay
// within 4 GiB, else fewer (at least one lr_horz block's worth).
static int vert_terms(const bf_plan *pl, int H, int W) {
    const size_t term_bytes = 4 * blocked_plane(H, W) * sizeof(float);
    const size_t budget = (size_t)4 << 30;
    const int nt = (int)pl->a32.size();
    const int cap = (int)std::max<size_t>(kHT, std::min<size_t>(kVMax, budget / term_bytes));
    return std::min(nt, cap);
}

// Q/P slot pairs: one per lr_horz term group of the largest lr_vert launch.
static int horz_slots(const bf_plan *pl, int H, int W) {
    return (vert_terms(pl, H, W) + kHT - 1) / kHT;
}

size_t large_workspace(const bf_plan *pl, int H, int W) {
    const size_t planes = 4 * (size_t)vert_terms(pl, H, W) + 2 * (size_t)horz_slots(pl, H, W) + 1;
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
    const int n_slots = horz_slots(pl, H, W);
    const size_t plane = blocked_plane(H, W);
    p.Vt = reinterpret_cast<float *>(base);
    p.Acc = p.Vt + (size_t)4 * gv_max * plane;
    p.ft = p.Acc + (size_t)2 * n_slots * plane;
    const int RS = ring_size(p.r);
    const size_t sm_v = sizeof(float) * (size_t)kVCols * (RS + kChunk);
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

    // lr_vert's bands (multiples of kChunk rows): as many as one wave of resident
    // blocks holds (a partial second wave costs a whole band's time), at
    // least 12r long (the 6r warm-up at most half a band).
    const int min_band = 12 * p.r;
    const int ncb = (W + kVCols - 1) / kVCols;
    const int zb_max = (gv_max + kVB - 1) / kVB;
    const int nbh_max = std::max(1, std::min(resident_vert / (ncb * zb_max), H / min_band));
    p.band_h = ((H + nbh_max - 1) / nbh_max + kChunk - 1) / kChunk * kChunk;
    const int nbh = (H + p.band_h - 1) / p.band_h;
    const int nyb2 = (p.nyb + 1) / 2;
    // lr_horz: resident blocks as many as fit the SMs -- for large r (the
    // prefetching variant) only as many as keep the columns each lane reads
    // back (3L of them, 8 bytes each) within kHorzL2Bytes of L2.  Bands of
    // columns only add warm-up, so there are just enough of them for every
    // resident block to have an item when the terms are few.
    // The prefetching variant needs enough items to fill its grid; with few
    // terms the other one, two blocks per SM over more bands, does better.
    const size_t lag_bytes = (size_t)64 * kHT * 8 * 3 * (size_t)L_of(p.r);
    const int items0 = nyb2 * ((std::min(nt, gv_max) + kHT - 1) / kHT);
    int per_sm_h = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_h, lr_horz<true>, 64 * kHT, 0);
    if (e != cudaSuccess) return e;
    const size_t pf_grid =
        std::min((size_t)n_sm * std::max(1, per_sm_h), kHorzL2Bytes / lag_bytes);
    const bool pf = p.r >= kHorzPrefetchR && (size_t)items0 >= pf_grid;
    auto kh = pf ? lr_horz<true> : lr_horz<false>;
    if (!pf) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_h, kh, 64 * kHT, 0);
        if (e != cudaSuccess) return e;
    }
    const int horz_grid = (int)std::max<size_t>(
        1, pf ? pf_grid : (size_t)n_sm * std::max(1, per_sm_h));
    const int nbw_max = std::max(1, std::min(horz_grid / items0, W / min_band));
    p.band_w = ((W + nbw_max - 1) / nbw_max + 7) / 8 * 8;
    const int nbw = (W + p.band_w - 1) / p.band_w;

    const int esz = img.dtype == 0 ? 4 : 1;
    for (int ch = 0; ch < img.C; ++ch) {
        p.in = reinterpret_cast<const char *>(img.in) + (long long)ch * img.in_z * esz;
        dim3 gt((W + 31) / 32, (H + 31) / 32);
        kt<<<gt, dim3(32, 8), 0, s>>>(p);
        for (int m0 = 0; m0 < nt; m0 += gv_max) {
            // terms [m0, m0 + nv): one lr_vert launch, then one lr_horz launch
            const int nv = std::min(gv_max, nt - m0);
            p.n_terms = nv;
            for (int g = 0; g < kVMax; ++g) {
                const int m = m0 + std::min(g, nv - 1);
                p.tv[g] = pl->turns32[m];
                p.th[g] = pl->turns32[m];
                p.ah[g] = pl->a32[m];
            }
            p.first = m0 == 0;
            dim3 gv(ncb, nbh, (nv + kVB - 1) / kVB);
            kv<<<gv, kVCols * kVB, sm_v, s>>>(p);
            const int items = nyb2 * nbw * ((nv + kHT - 1) / kHT);
            kh<<<std::min(items, horz_grid), 64 * kHT, 0, s>>>(p);
        }
        dim3 gf((W + 31) / 32, (H + 31) / 32);
        lr_final<<<gf, dim3(32, 8), 0, s>>>(
            p.Acc, n_slots, img.out + (long long)ch * img.out_z,
            img.q_out ? img.q_out + (long long)ch * img.out_z : nullptr, H, W, img.out_px,
            img.q_scale);
    }
    return cudaGetLastError();
}


// ---- recursive Gaussian: scratch and launches -------------------------------

static size_t rg_plane(const bf_plan *pl, int H, int W) {  // float2 elements
    const int P = pl->rg_P;
    const size_t nybe = (size_t)(H + P + kYB - 1) / kYB;
    const size_t We = (size_t)(W + P + kChunkH - 1) / kChunkH * kChunkH;
    return nybe * kYB * We;
}

static int rg_terms(const bf_plan *pl, int H, int W) {
    const size_t term_bytes = 2 * rg_plane(pl, H, W) * sizeof(float2);
    const size_t budget = (size_t)4 << 30;
    const int nt = (int)pl->a32.size();
    const int cap = (int)std::max<size_t>(kHT, std::min<size_t>(kVMax, budget / term_bytes));
    return std::min(nt, cap);
}

size_t recursive_workspace(const bf_plan *pl, int H, int W) {
    const int m = rg_terms(pl, H, W);
    const size_t slots = (size_t)(m + kHT - 1) / kHT;
    return (size_t)m * 2 * rg_plane(pl, H, W) * sizeof(float2) +
           (2 * slots + 1) * blocked_plane(H, W) * sizeof(float) + 256;
}

cudaError_t launch_recursive(const bf_plan *pl, const BfImage &img, void *ws, cudaStream_t s) {
    const int H = img.H, W = img.W;
    const int nt = (int)pl->a32.size();
    const int gv_max = rg_terms(pl, H, W);
    const int n_slots = (gv_max + kHT - 1) / kHT;
    char *base = reinterpret_cast<char *>(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    RgParams p{};
    p.in_stride = img.in_row_stride;
    p.dtype = img.dtype;
    p.in_px = img.in_px;
    p.H = H;
    p.W = W;
    p.P = pl->rg_P;
    p.We = (W + p.P + kChunkH - 1) / kChunkH * kChunkH;
    p.nybe = (H + p.P + kYB - 1) / kYB;
    p.nyb = (H + kYB - 1) / kYB;
    p.cB = (float)pl->rg[0];
    p.cD1 = (float)(pl->rg[2] + pl->rg[3]);
    p.cD2 = (float)pl->rg[3];
    const size_t fplane = blocked_plane(H, W);
    p.Vt = reinterpret_cast<float *>(base);
    p.Acc = p.Vt + (size_t)gv_max * 2 * rg_plane(pl, H, W) * 2;
    float *ft = p.Acc + (size_t)2 * n_slots * fplane;
    p.ft = ft;
    LrParams lp{};  // for the shared transpose and final kernels
    lp.in_stride = img.in_row_stride;
    lp.dtype = img.dtype;
    lp.in_px = img.in_px;
    lp.H = H;
    lp.W = W;
    lp.ft = ft;
    auto kv = img.dtype == 0 ? rg_vert<0> : rg_vert<1>;
    auto kt = img.dtype == 0 ? lr_transpose<0> : lr_transpose<1>;
    const int ncb = (W + kVCols - 1) / kVCols;
    const int esz = img.dtype == 0 ? 4 : 1;
    for (int ch = 0; ch < img.C; ++ch) {
        p.in = reinterpret_cast<const char *>(img.in) + (long long)ch * img.in_z * esz;
        lp.in = p.in;
        dim3 gt((W + 31) / 32, (H + 31) / 32);
        kt<<<gt, dim3(32, 8), 0, s>>>(lp);
        for (int m0 = 0; m0 < nt; m0 += gv_max) {
            const int nv = std::min(gv_max, nt - m0);
            p.n_terms = nv;
            for (int g = 0; g < kVMax; ++g) {
                const int m = m0 + std::min(g, nv - 1);
                p.tv[g] = pl->turns32[m];
                p.ah[g] = pl->a32[m];
            }
            p.first = m0 == 0;
            dim3 gv(ncb, 1, (nv + kVB - 1) / kVB);
            kv<<<gv, kVCols * kVB, 0, s>>>(p);
            dim3 gh((p.nyb + 1) / 2, 1, (nv + kHT - 1) / kHT);
            rg_horz<<<gh, 64 * kHT, 0, s>>>(p);
        }
        dim3 gf((W + 31) / 32, (H + 31) / 32);
        lr_final<<<gf, dim3(32, 8), 0, s>>>(
            p.Acc, n_slots, img.out + (long long)ch * img.out_z,
            img.q_out ? img.q_out + (long long)ch * img.out_z : nullptr, H, W, img.out_px,
            img.q_scale);
    }
    return cudaGetLastError();
}

}  // namespace bf

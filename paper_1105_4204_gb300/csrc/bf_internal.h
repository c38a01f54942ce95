// Internal declarations shared by the host side and the kernels of libbf.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/bf.h"

// Largest degree the kernels accept; terms = ceil(N/2) (+1 for even N).
#define BF_MAX_N 1024
#define BF_MAX_TERMS 520
// Largest 1-D support half-width of a truncated Gaussian handled by taps.
#define BF_MAX_TAPS_R 32
// Tallest image: the tile kernels put the row tiles (32 rows or more) on
// gridDim.y, which is at most 65535.
#define BF_MAX_ROWS (65535 * 32)

struct bf_plan {
    double sigma_s = 0, sigma_r = 0, T = 0;
    int kind = 0;          // bf_spatial_kind
    int N = 1;             // degree
    int passes = 3;        // box passes
    int r_box = 0;         // box half-width
    int R = 0;             // support half-width per axis
    double achieved_sigma = 0;
    // Terms in accumulation order (smallest weight first, omega = 0 last).
    std::vector<double> a, omega;
    std::vector<float> a32, turns32;  // FP32 weight, omega / (2 pi) in turns per gray level
    bool has_center = false;
    std::vector<double> w1;           // 1-D taps, 2R+1, unit sum
    std::vector<float> w1f;
    // Normaliser scale: the kernels filter the box unnormalised (integer
    // weights) since the ratio P/Q does not depend on a common scale.
    float q_scale = 1.f;
    // A general cosine polynomial of Section 2.2 (bf_plan_create_cosine):
    // phi(s) = sum_n a_n cos(n gamma s); sigma_r and T are then 0.
    bool cosine = false;
    double gamma = 0.0;
    // Recursive Gaussian (kind 2): B, b1/b0, b2/b0, b3/b0 and the extension P.
    double rg[4] = {0, 0, 0, 0};
    int rg_P = 0;
};

// Per-launch term table, passed by value as a kernel parameter (constant bank).
struct BfTerms {
    int n_terms;
    float a[BF_MAX_TERMS];
    float t[BF_MAX_TERMS];  // turns per gray level
};

struct BfTaps {
    float w[2 * BF_MAX_TAPS_R + 1];
    float2 w2[2 * BF_MAX_TAPS_R + 1];  // the same taps, each duplicated into a pair
};

// One launch covers C planes (z): interleaved channels of one image
// (px_stride = C, z_stride = 1) or a stack of single-channel images
// (px_stride = 1, z_stride = image size).
struct BfImage {
    const void *in;
    float *out;
    float *q_out;
    long long in_row_stride;  // elements
    int H, W, C;
    int dtype;                // 0 f32, 1 u8
    float q_scale;
    int in_px, out_px;        // elements between horizontally adjacent pixels
    long long in_z, out_z;    // elements between consecutive planes z
};

namespace bf {

void set_error(const std::string &msg);
bf_status fail(bf_status st, const std::string &msg);
bf_status cuda_check(cudaError_t e, const char *what);

void fill_terms(const bf_plan *p, BfTerms *t);
void fill_taps(const bf_plan *p, BfTaps *t);
// Copies t->w into the paired taps t->w2.
void pair_taps(BfTaps *t);

// Launchers (return cudaGetLastError() of the launch).
// Fused tile kernel for the truncated Gaussian / small-radius box.
bool tile_supported(const bf_plan *p);
cudaError_t launch_tile_forward(const bf_plan *p, const BfImage &img, cudaStream_t s);

// Streaming sweeps for the 3-pass box with r > 8 (one image, its channels in
// turn) through a scratch buffer of large_workspace(p, H, W) bytes.
size_t large_workspace(const bf_plan *p, int H, int W);
cudaError_t launch_large_box(const bf_plan *p, const BfImage &img, void *ws, cudaStream_t s);
// The recursive Gaussian (kind 2): a vertical and a horizontal recursive
// sweep through a scratch buffer of recursive_workspace(p, H, W) bytes.
size_t recursive_workspace(const bf_plan *p, int H, int W);
cudaError_t launch_recursive(const bf_plan *p, const BfImage &img, void *ws, cudaStream_t s);

// Space-variant extension (one half-width per pixel, 0 <= r <= r_max <=
// sv_max_radius(hat)), C interleaved channels; the box (hat = 0) or the
// separable hat (hat = 1).
int sv_max_radius(int hat);
cudaError_t launch_space_variant(const bf_plan *pl, const void *in, int dtype,
                                 long long row_stride, const int *radius, int r_max, int hat,
                                 float *out, int H, int W, int C, cudaStream_t s);

}  // namespace bf

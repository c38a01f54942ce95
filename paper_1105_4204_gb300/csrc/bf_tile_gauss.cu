// Instantiations of the fused tile kernel for the truncated Gaussian.
// A support radius R is served by the smallest instantiated radius >= R with
// the taps centred and zero-padded; a zero tap adds exactly 0 in FP32, so the
// result equals the one a radius-R kernel would give.
#include "bf_tile.cuh"

namespace bf {

static const int kGaussRadii[] = {2, 4, 6, 9, 12, 15, 18, 24};

int gauss_tile_radius(int R) {
    for (int r : kGaussRadii)
        if (r >= R) return r;
    return -1;
}

// Tile shapes by id: 0 = 32 x 64 tiles, 16-pixel segments; 1 (small radii
// only) = 32 x 96 tiles, 24-pixel segments (more phase-1 work items per block
// and less halo, at the cost of registers); 2 (radii >= 9) = 64 x 64 tiles,
// one 512-thread block per SM.  Fills ids, returns their number.
int gauss_tile_shape_ids(int R, int *ids) {
    const int Ri = gauss_tile_radius(R);
    int n = 0;
    ids[n++] = 0;
    if (Ri > 0 && Ri <= 9) ids[n++] = 1;
    if (Ri >= 9) ids[n++] = 2;
    return n;
}

cudaError_t launch_tile_gauss(const bf_plan *pl, const BfImage &img, cudaStream_t s, int shape,
                              int split) {
    const int Ri = gauss_tile_radius(pl->R);
    TileParams prm;
    prm.img = img;
    prm.split = split;
    fill_terms(pl, &prm.terms);
    for (int k = 0; k < 2 * BF_MAX_TAPS_R + 1; ++k) prm.taps.w[k] = 0.f;
    for (int k = 0; k < 2 * pl->R + 1; ++k) prm.taps.w[k + Ri - pl->R] = pl->w1f[k];
    pair_taps(&prm.taps);
    if (shape == 1) {
        switch (Ri) {
            case 2: return launch_tile<0, 2, 32, 96, 24>(prm, s);
            case 4: return launch_tile<0, 4, 32, 96, 24>(prm, s);
            case 6: return launch_tile<0, 6, 32, 96, 24>(prm, s);
            case 9: return launch_tile<0, 9, 32, 96, 24>(prm, s);
            default: break;
        }
    }
    if (shape == 2) {
        switch (Ri) {
            case 9: return launch_tile<0, 9, 64, 64, 16>(prm, s);
            case 12: return launch_tile<0, 12, 64, 64, 16>(prm, s);
            case 15: return launch_tile<0, 15, 64, 64, 16>(prm, s);
            case 18: return launch_tile<0, 18, 64, 64, 16>(prm, s);
            case 24: return launch_tile<0, 24, 64, 64, 16>(prm, s);
            default: break;
        }
    }
    switch (Ri) {
        case 2: return launch_tile<0, 2, 32, 64, 16>(prm, s);
        case 4: return launch_tile<0, 4, 32, 64, 16>(prm, s);
        case 6: return launch_tile<0, 6, 32, 64, 16>(prm, s);
        case 9: return launch_tile<0, 9, 32, 64, 16>(prm, s);
        case 12: return launch_tile<0, 12, 32, 64, 16>(prm, s);
        case 15: return launch_tile<0, 15, 32, 64, 16>(prm, s);
        case 18: return launch_tile<0, 18, 32, 64, 16>(prm, s);
        case 24: return launch_tile<0, 24, 32, 64, 16>(prm, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bf


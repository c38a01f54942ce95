// Instantiations of the fused tile kernel for the 3-pass iterated box.
#include "bf_tile.cuh"

namespace bf {

int box_tile_max_r() { return 8; }

// Tile shapes by id: 0 = 32 x 64 tiles, 16-pixel segments (two or three
// blocks per SM); 1 (r <= 4) = 32 x 96 tiles, 24-pixel segments; 2 (r >= 3) =
// 64 x 64 tiles, 16-pixel segments, one 512-thread block per SM (less halo
// per output at the cost of occupancy); 3 (r >= 7) = 64 x 64 tiles, 32-pixel
// segments, one 256-thread block per SM (also less warm-up per segment, at
// half the warps; measured 4 % faster than id 0 at r = 8 on 2048 x 2048,
// slower below r = 7).  Fills ids, returns their number.
int box_tile_shape_ids(int r, int *ids) {
    int n = 0;
    ids[n++] = 0;
    if (r >= 1 && r <= 4) ids[n++] = 1;
    if (r >= 3 && r <= 8) ids[n++] = 2;
    if (r >= 7 && r <= 8) ids[n++] = 3;
    return n;
}

cudaError_t launch_tile_box_long_segments(int r, const TileParams &prm, cudaStream_t s);

cudaError_t launch_tile_box(const bf_plan *pl, const BfImage &img0, cudaStream_t s, int shape,
                            int split) {
    TileParams prm;
    prm.img = img0;
    prm.split = split;
    fill_terms(pl, &prm.terms);
    for (int k = 0; k < 2 * BF_MAX_TAPS_R + 1; ++k) prm.taps.w[k] = 0.f;
    pair_taps(&prm.taps);
    if (shape == 1) {
        switch (pl->r_box) {
            case 1: return launch_tile<1, 1, 32, 96, 24>(prm, s);
            case 2: return launch_tile<1, 2, 32, 96, 24>(prm, s);
            case 3: return launch_tile<1, 3, 32, 96, 24>(prm, s);
            case 4: return launch_tile<1, 4, 32, 96, 24>(prm, s);
            default: break;
        }
    }
    if (shape == 3) return launch_tile_box_long_segments(pl->r_box, prm, s);
    if (shape == 2) {
        switch (pl->r_box) {
            case 3: return launch_tile<1, 3, 64, 64, 16>(prm, s);
            case 4: return launch_tile<1, 4, 64, 64, 16>(prm, s);
            case 5: return launch_tile<1, 5, 64, 64, 16>(prm, s);
            case 6: return launch_tile<1, 6, 64, 64, 16>(prm, s);
            case 7: return launch_tile<1, 7, 64, 64, 16>(prm, s);
            case 8: return launch_tile<1, 8, 64, 64, 16>(prm, s);
            default: break;
        }
    }
    switch (pl->r_box) {
        case 1: return launch_tile<1, 1, 32, 64, 16>(prm, s);
        case 2: return launch_tile<1, 2, 32, 64, 16>(prm, s);
        case 3: return launch_tile<1, 3, 32, 64, 16>(prm, s);
        case 4: return launch_tile<1, 4, 32, 64, 16>(prm, s);
        case 5: return launch_tile<1, 5, 32, 64, 16>(prm, s);
        case 6: return launch_tile<1, 6, 32, 64, 16>(prm, s);
        case 7: return launch_tile<1, 7, 32, 64, 16>(prm, s);
        case 8: return launch_tile<1, 8, 32, 64, 16>(prm, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bf

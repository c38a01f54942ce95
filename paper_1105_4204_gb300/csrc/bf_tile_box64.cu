// Instantiations of the fused tile kernel for the 3-pass box with 64 x 64
// tiles and 32-pixel row segments (tile shape id 3), in their own translation
// unit so that the library's objects compile in parallel.
#include "bf_tile.cuh"

namespace bf {

cudaError_t launch_tile_box_long_segments(int r, const TileParams &prm, cudaStream_t s) {
    switch (r) {
        case 7: return launch_tile<1, 7, 64, 64, 32>(prm, s);
        case 8: return launch_tile<1, 8, 64, 64, 32>(prm, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bf

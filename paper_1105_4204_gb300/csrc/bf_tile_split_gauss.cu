// Term-split (thread-block cluster) instantiations of the fused tile kernel
// for the truncated Gaussian (the box's are in bf_tile_split.cu):
// a tile's terms cut into groups, one block per group, the groups reduced in
// group order through distributed shared memory.  Small images use them on
// the 32-row tiles; every shape has them so that any configuration can be
// pinned.  In their own translation unit so that the library's objects
// compile in parallel.
#include "bf_tile.cuh"

namespace bf {

template <int KIND, int RAD, int TH, int TW, int TWT>
cudaError_t launch_tile_cluster(const TileParams &prm, cudaStream_t s) {
    return launch_tile_cluster_impl<KIND, RAD, TH, TW, TWT>(prm, s);
}

#define BF_SPLIT(kind, r, th, tw, twt)                                                  \
    template cudaError_t launch_tile_cluster<kind, r, th, tw, twt>(const TileParams &, \
                                                                   cudaStream_t);

// truncated Gaussian: 32 x 64 tiles (every instantiated radius), 32 x 96
// (R <= 9), 64 x 64 (R >= 9)
BF_SPLIT(0, 2, 32, 64, 16) BF_SPLIT(0, 4, 32, 64, 16) BF_SPLIT(0, 6, 32, 64, 16)
BF_SPLIT(0, 9, 32, 64, 16) BF_SPLIT(0, 12, 32, 64, 16) BF_SPLIT(0, 15, 32, 64, 16)
BF_SPLIT(0, 18, 32, 64, 16) BF_SPLIT(0, 24, 32, 64, 16)
BF_SPLIT(0, 2, 32, 96, 24) BF_SPLIT(0, 4, 32, 96, 24) BF_SPLIT(0, 6, 32, 96, 24)
BF_SPLIT(0, 9, 32, 96, 24)
BF_SPLIT(0, 9, 64, 64, 16) BF_SPLIT(0, 12, 64, 64, 16) BF_SPLIT(0, 15, 64, 64, 16)
BF_SPLIT(0, 18, 64, 64, 16) BF_SPLIT(0, 24, 64, 64, 16)

#undef BF_SPLIT

}  // namespace bf

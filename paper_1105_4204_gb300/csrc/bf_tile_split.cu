// Term-split (thread-block cluster) instantiations of the fused tile kernel
// for the 3-pass box (the Gaussian's are in bf_tile_split_gauss.cu):
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

// 3-pass box: 32 x 64 tiles (r = 1 .. 8), 32 x 96 (r = 1 .. 4), 64 x 64 (r = 3 .. 8),
// 64 x 64 with 32-pixel segments (r = 7, 8)
BF_SPLIT(1, 1, 32, 64, 16) BF_SPLIT(1, 2, 32, 64, 16) BF_SPLIT(1, 3, 32, 64, 16)
BF_SPLIT(1, 4, 32, 64, 16) BF_SPLIT(1, 5, 32, 64, 16) BF_SPLIT(1, 6, 32, 64, 16)
BF_SPLIT(1, 7, 32, 64, 16) BF_SPLIT(1, 8, 32, 64, 16)
BF_SPLIT(1, 1, 32, 96, 24) BF_SPLIT(1, 2, 32, 96, 24) BF_SPLIT(1, 3, 32, 96, 24)
BF_SPLIT(1, 4, 32, 96, 24)
BF_SPLIT(1, 3, 64, 64, 16) BF_SPLIT(1, 4, 64, 64, 16) BF_SPLIT(1, 5, 64, 64, 16)
BF_SPLIT(1, 6, 64, 64, 16) BF_SPLIT(1, 7, 64, 64, 16) BF_SPLIT(1, 8, 64, 64, 16)
BF_SPLIT(1, 7, 64, 64, 32) BF_SPLIT(1, 8, 64, 64, 32)

#undef BF_SPLIT

}  // namespace bf

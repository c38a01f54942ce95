// Instantiations of the fused backward kernel for the 3-pass iterated box
// (a translation unit of its own so that it compiles beside the Gaussian ones).
#include "bf_bwd.cuh"

namespace bf {

cudaError_t launch_bwd_box(int r, const BwdParams &prm, int count, cudaStream_t s) {
    switch (r) {
        case 1: return launch_bwd<1, 1, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s);
        case 2: return launch_bwd<1, 2, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s);
        case 3: return launch_bwd<1, 3, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s);
        case 4: return launch_bwd<1, 4, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s);
        case 5: return launch_bwd<1, 5, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s);
        case 6: return launch_bwd<1, 6, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s);
        case 7: return launch_bwd<1, 7, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s);
        case 8: return launch_bwd<1, 8, kBwdTH, kBwdTW, kBwdTWT>(prm, count, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bf

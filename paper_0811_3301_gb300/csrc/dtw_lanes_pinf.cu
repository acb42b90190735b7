// Warp-path band-DTW kernels for p = infinity.
#include "dtw_launch.cuh"

namespace dtwk {

cudaError_t launch_dtw_lanes_pinf(const DtwJob &j, const DtwGeom &g, LanesShape ls, cudaStream_t s) {
    return launch_dtw_lanes_pt<0>(j, g, ls, s);
}

}  // namespace dtwk

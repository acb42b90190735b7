// Warp-path band-DTW kernels for p = 4.
#include "dtw_launch.cuh"

namespace dtwk {

cudaError_t launch_dtw_lanes_p4(const DtwJob &j, const DtwGeom &g, LanesShape ls, cudaStream_t s) {
    return launch_dtw_lanes_pt<4>(j, g, ls, s);
}

}  // namespace dtwk

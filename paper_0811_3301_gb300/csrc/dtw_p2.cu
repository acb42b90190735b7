// Band-DTW kernels (register and wide thread paths) for p = 2.
#include "dtw_launch.cuh"

namespace dtwk {

cudaError_t launch_dtw_p2(const DtwJob &j, const DtwGeom &g, cudaStream_t s) { return launch_dtw_pt<2>(j, g, s); }
cudaError_t launch_dtw_phase_p2(const DtwJob &j, const DtwGeom &g, cudaStream_t s) {
    return launch_dtw_phase_pt<2>(j, g, s);
}

}  // namespace dtwk

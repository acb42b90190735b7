// Band-DTW kernels (register and wide thread paths) for p = infinity.
#include "dtw_launch.cuh"

namespace dtwk {

cudaError_t launch_dtw_pinf(const DtwJob &j, const DtwGeom &g, cudaStream_t s) { return launch_dtw_pt<0>(j, g, s); }
cudaError_t launch_dtw_phase_pinf(const DtwJob &j, const DtwGeom &g, cudaStream_t s) {
    return launch_dtw_phase_pt<0>(j, g, s);
}

}  // namespace dtwk

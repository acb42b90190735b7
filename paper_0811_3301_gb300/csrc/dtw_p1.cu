// Band-DTW kernels (register and wide thread paths) for p = 1.
#include "dtw_launch.cuh"

namespace dtwk {

cudaError_t launch_dtw_p1(const DtwJob &j, const DtwGeom &g, cudaStream_t s) { return launch_dtw_pt<1>(j, g, s); }
cudaError_t launch_dtw_phase_p1(const DtwJob &j, const DtwGeom &g, cudaStream_t s) {
    return launch_dtw_phase_pt<1>(j, g, s);
}

}  // namespace dtwk

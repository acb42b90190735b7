// Warp-path DTW instantiations for p = 2 (slots per lane CL).
#include "dtw_lanes.cuh"

namespace dtwk {

cudaError_t launch_dtw_lanes_p2(const DtwJob &j, const DtwGeom &g, int cl, cudaStream_t s) {
    if (j.npairs <= 0) return cudaSuccess;
    const int n = j.n;
    const int w = j.w < n - 1 ? j.w : n - 1;
    // every query-copy index the lanes read: padl - w >= 0 (row 0, slot 0) up to
    // padl + n - 1 + w + cl - 1 (row n-1, top slot of the band's last lane)
    if (g.padl < w || (int64_t)g.padl + n + w + cl > (int64_t)j.qc.ylen || 2 * w + 1 > 32 * cl)
        return cudaErrorInvalidValue;
    const int64_t warps = (j.npairs + 1) / 2;
#define DTW_LANES_CASE(CC)                                                            \
    case CC: {                                                                        \
        auto kern = k_dtw_lanes<CC, 2>;                                            \
        int per_sm = 0;                                                               \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDtwThreads, 0); \
        if (per_sm < 1) per_sm = 1;                                                   \
        const int64_t full = (int64_t)per_sm * device_sm_count();                     \
        int64_t need = (warps + (kDtwThreads / 32) - 1) / (kDtwThreads / 32);         \
        if (need < 1) need = 1;                                                       \
        kern<<<(int)(need < full ? need : full), kDtwThreads, 0, s>>>(j);             \
        break;                                                                        \
    }
    switch (cl) {
        DTW_LANES_CASE(2) DTW_LANES_CASE(3) DTW_LANES_CASE(4) DTW_LANES_CASE(5) DTW_LANES_CASE(6)
        DTW_LANES_CASE(7) DTW_LANES_CASE(8) DTW_LANES_CASE(10) DTW_LANES_CASE(12) DTW_LANES_CASE(13)
        DTW_LANES_CASE(16) DTW_LANES_CASE(20) DTW_LANES_CASE(24) DTW_LANES_CASE(32)
        default: return cudaErrorInvalidValue;
    }
#undef DTW_LANES_CASE
    return cudaGetLastError();
}

}  // namespace dtwk

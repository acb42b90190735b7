// Warp-path DTW instantiations for p = 1 (lanes per pair G, slots per lane CL).
#include "dtw_lanes.cuh"

namespace dtwk {

cudaError_t launch_dtw_lanes_p1(const DtwJob &j, const DtwGeom &g, LanesShape ls, cudaStream_t s) {
    if (j.npairs <= 0) return cudaSuccess;
    const int n = j.n;
    const int w = j.w < n - 1 ? j.w : n - 1;
    // every query-copy index the lanes read: padl - w >= 0 (row 0, slot 0) up to
    // padl + n - 1 + w + cl - 1 (row n-1, top slot of the band's last lane)
    if (g.padl < w || (int64_t)g.padl + n + w + ls.cl > (int64_t)j.qc.ylen || 2 * w + 1 > ls.g * ls.cl)
        return cudaErrorInvalidValue;
    const int64_t warps = (j.npairs + 2 * (32 / ls.g) - 1) / (2 * (32 / ls.g));
#define DTW_LANES_CASE(GG, CC)                                                        \
    if (ls.g == GG && ls.cl == CC) {                                                  \
        auto kern = k_dtw_lanes<CC, GG, 1>;                                        \
        int per_sm = 0;                                                               \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDtwThreads, 0); \
        if (per_sm < 1) per_sm = 1;                                                   \
        const int64_t full = (int64_t)per_sm * device_sm_count();                     \
        int64_t need = (warps + (kDtwThreads / 32) - 1) / (kDtwThreads / 32);         \
        if (need < 1) need = 1;                                                       \
        kern<<<(int)(need < full ? need : full), kDtwThreads, 0, s>>>(j);             \
        return cudaGetLastError();                                                    \
    }
    DTW_LANES_CASE(16, 4) DTW_LANES_CASE(16, 7) DTW_LANES_CASE(16, 10) DTW_LANES_CASE(16, 13)
    DTW_LANES_CASE(16, 16) DTW_LANES_CASE(16, 20) DTW_LANES_CASE(16, 26) DTW_LANES_CASE(16, 32)
    DTW_LANES_CASE(32, 2) DTW_LANES_CASE(32, 3) DTW_LANES_CASE(32, 4) DTW_LANES_CASE(32, 5)
    DTW_LANES_CASE(32, 6) DTW_LANES_CASE(32, 7) DTW_LANES_CASE(32, 8) DTW_LANES_CASE(32, 10)
    DTW_LANES_CASE(32, 13) DTW_LANES_CASE(32, 16) DTW_LANES_CASE(32, 20) DTW_LANES_CASE(32, 24)
    DTW_LANES_CASE(32, 32)
#undef DTW_LANES_CASE
    return cudaErrorInvalidValue;
}

}  // namespace dtwk

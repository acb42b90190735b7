// DTW kernel instantiations for p = 1 (band widths of the register and wide paths).
#include "dtw_kernels.cuh"

namespace dtwk {

namespace {
template <typename K>
int blocks_for(K kernel, int64_t warps_needed) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kDtwThreads, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t full = (int64_t)per_sm * device_sm_count();
    int64_t need = (warps_needed + (kDtwThreads / 32) - 1) / (kDtwThreads / 32);
    if (need < 1) need = 1;
    return (int)(need < full ? need : full);
}
}  // namespace

cudaError_t launch_dtw_p1(const DtwJob &j, const DtwGeom &g, cudaStream_t s) {
    if (j.npairs <= 0) return cudaSuccess;
    const bool many = j.lanes == 2 || (j.npairs_dev == nullptr && j.npairs >= 65536);
    const LanesShape ls = dtw_lanes_shape(j.n, j.w, many);
    // one query per pair: a thread per pair would read its own band-wide query
    // window every row, the warp path one value per row and lane
    const bool per_pair_wide = j.per_pair_y && j.n >= 64 && 2 * j.w + 1 > 32;
    if ((j.lanes || g.wide || per_pair_wide) && ls.cl > 0) return launch_dtw_lanes_p1(j, g, ls, s);
    if (!g.wide && g.C <= kDtwGroupMaxC) {
        const int64_t warps = (j.npairs + 31) / 32;
        const bool xvec = (j.n % 4 == 0) && ((reinterpret_cast<uintptr_t>(j.db) & 15) == 0);
        // bands of 10 % of the common lengths get a compile-time bottom padding:
        // (C, e) = (16, 3) w = 6, (32, 7) w = 12, (48, 11) w = 18, (64, 13) w = 25
#define DTW_REG4_FIXED(CC, EE)                                                        \
    if (g.C == CC && g.e == EE) {                                                     \
        auto kern = k_dtw_reg4<CC, 1, EE>;                                          \
        kern<<<blocks_for(kern, warps), kDtwThreads, 0, s>>>(j, g.e, g.wl, xvec);     \
        return cudaGetLastError();                                                    \
    }
        DTW_REG4_FIXED(16, 3) DTW_REG4_FIXED(32, 7) DTW_REG4_FIXED(48, 11) DTW_REG4_FIXED(64, 13)
#undef DTW_REG4_FIXED
#define DTW_REG4_CASE(CC)                                                             \
    case CC: {                                                                        \
        auto kern = k_dtw_reg4<CC, 1, -1>;                                          \
        kern<<<blocks_for(kern, warps), kDtwThreads, 0, s>>>(j, g.e, g.wl, xvec);     \
        break;                                                                        \
    }
        switch (g.C) {
            DTW_REG4_CASE(16) DTW_REG4_CASE(32) DTW_REG4_CASE(48) DTW_REG4_CASE(64)
            default: return cudaErrorInvalidValue;
        }
#undef DTW_REG4_CASE
    } else if (!g.wide) {
        const int64_t warps = (j.npairs + 31) / 32;
#define DTW_REG_CASE(CC)                                                              \
    case CC: {                                                                        \
        auto kern = k_dtw_reg<CC, 1>;                                                \
        kern<<<blocks_for(kern, warps), kDtwThreads, 0, s>>>(j, g.e, g.wl);           \
        break;                                                                        \
    }
        switch (g.C) {
            DTW_REG_CASE(16) DTW_REG_CASE(32) DTW_REG_CASE(48) DTW_REG_CASE(64)
            DTW_REG_CASE(80) DTW_REG_CASE(96) DTW_REG_CASE(112) DTW_REG_CASE(128)
            DTW_REG_CASE(144) DTW_REG_CASE(160) DTW_REG_CASE(176) DTW_REG_CASE(192)
            DTW_REG_CASE(208)
            default: return cudaErrorInvalidValue;
        }
#undef DTW_REG_CASE
    } else {
        const int64_t warps = j.npairs;
#define DTW_WIDE_CASE(CC)                                                             \
    case CC: {                                                                        \
        auto kern = k_dtw_wide<CC, 1>;                                               \
        kern<<<blocks_for(kern, warps), kDtwThreads, 0, s>>>(j);                      \
        break;                                                                        \
    }
        switch (g.cl) {
            DTW_WIDE_CASE(8) DTW_WIDE_CASE(16) DTW_WIDE_CASE(32) DTW_WIDE_CASE(64)
            default: return cudaErrorInvalidValue;
        }
#undef DTW_WIDE_CASE
    }
    return cudaGetLastError();
}

}  // namespace dtwk

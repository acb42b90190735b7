// Launchers of the band-DTW kernels for one cost exponent P (1, 2, 4, or 0
// for p = infinity): the warp path and the register / wide thread paths,
// with the band widths they are compiled for.  Each p has its own translation
// units (dtw_p*.cu, dtw_lanes_p*.cu) so that they compile in parallel.
#pragma once
#include "dtw_lanes.cuh"
#include "dtw_wave.cuh"

namespace dtwk {

namespace launch_detail {
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
}  // namespace launch_detail

template <int P>
cudaError_t launch_dtw_lanes_pt(const DtwJob &j, const DtwGeom &g, LanesShape ls, cudaStream_t s) {
    if (j.npairs <= 0) return cudaSuccess;
    const int n = j.n;
    const int w = j.w < n - 1 ? j.w : n - 1;
    // bands of 10 % of 1448 and of 20 % (or 10 % of 2048): the one-row-per-step
    // wavefront (dtw_wave.cuh), one pair per 32 lanes, compile-time padding;
    // lanes == 2 (two 16-lane groups per warp) keeps the two-steps-per-row kernel
    if (j.lanes != 2) {
        const int bw = 2 * w + 1;
#define DTW_WAVE_CASE(CC, GG, EE)                                                                 \
    if (bw + (EE) == (CC) * (GG)) {                                                               \
        const int wl = w + (EE);                                                                  \
        /* query-copy indices read: padl - wl (row 0, slot 0) .. padl + n - 1 + w */             \
        if (g.padl < wl || (int64_t)g.padl + n + w > (int64_t)j.qc.ylen) return cudaErrorInvalidValue; \
        auto kern = k_dtw_wave<CC, GG, P, EE>;                                                    \
        const int64_t warps = (j.npairs + (32 / (GG)) - 1) / (32 / (GG));                         \
        kern<<<launch_detail::blocks_for(kern, warps), kDtwThreads, 0, s>>>(j);                   \
        return cudaGetLastError();                                                                \
    }
        DTW_WAVE_CASE(13, 32, 7) DTW_WAVE_CASE(10, 32, 31)
#undef DTW_WAVE_CASE
    }
    // every query-copy index the lanes read: padl - w >= 0 (row 0, slot 0) up to
    // padl + n - 1 + w + cl - 1 (row n-1, top slot of the band's last lane)
    if (g.padl < w || (int64_t)g.padl + n + w + ls.cl > (int64_t)j.qc.ylen || 2 * w + 1 > ls.g * ls.cl)
        return cudaErrorInvalidValue;
    const int64_t warps = (j.npairs + 2 * (32 / ls.g) - 1) / (2 * (32 / ls.g));
#define DTW_LANES_CASE(GG, CC)                                                        \
    if (ls.g == GG && ls.cl == CC) {                                                  \
        auto kern = k_dtw_lanes<CC, GG, P>;                                        \
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




template <int P>
cudaError_t launch_dtw_pt(const DtwJob &j, const DtwGeom &g, cudaStream_t s) {
    if (j.npairs <= 0) return cudaSuccess;
    const bool many = j.lanes == 2 || (j.npairs_dev == nullptr && j.npairs >= 65536);
    const LanesShape ls = dtw_lanes_shape(j.n, j.w, many);
    // one query per pair: a thread per pair would read its own band-wide query
    // window every row, the warp path one value per row and lane
    const bool per_pair_wide = j.per_pair_y && j.n >= 64 && 2 * j.w + 1 > 32;
    if ((j.lanes || g.wide || per_pair_wide) && ls.cl > 0) return launch_dtw_lanes_pt<P>(j, g, ls, s);
    if (!g.wide && g.C <= kDtwGroupMaxC) {
        const int64_t warps = (j.npairs + 31) / 32;
        const bool xvec = (j.n % 4 == 0) && ((reinterpret_cast<uintptr_t>(j.db) & 15) == 0);
        // bands of 10 % of the common lengths get a compile-time bottom padding:
        // (C, e) = (16, 3) w = 6, (32, 7) w = 12, (48, 11) w = 18, (64, 13) w = 25
#define DTW_REG4_FIXED(CC, EE)                                                        \
    if (g.C == CC && g.e == EE) {                                                     \
        auto kern = k_dtw_reg4<CC, P, EE>;                                          \
        kern<<<launch_detail::blocks_for(kern, warps), kDtwThreads, 0, s>>>(j, g.e, g.wl, xvec);     \
        return cudaGetLastError();                                                    \
    }
        DTW_REG4_FIXED(16, 3) DTW_REG4_FIXED(32, 7) DTW_REG4_FIXED(48, 11) DTW_REG4_FIXED(64, 13)
#undef DTW_REG4_FIXED
#define DTW_REG4_CASE(CC)                                                             \
    case CC: {                                                                        \
        auto kern = k_dtw_reg4<CC, P, -1>;                                          \
        kern<<<launch_detail::blocks_for(kern, warps), kDtwThreads, 0, s>>>(j, g.e, g.wl, xvec);     \
        break;                                                                        \
    }
        switch (g.C) {
            DTW_REG4_CASE(16) DTW_REG4_CASE(32) DTW_REG4_CASE(48) DTW_REG4_CASE(64)
            default: return cudaErrorInvalidValue;
        }
#undef DTW_REG4_CASE
    } else if (!g.wide) {
        const int64_t warps = (j.npairs + 31) / 32;
        // bands of 10 % of the bucket lengths 724 ... 1448 get a compile-time
        // bottom padding and two rows per step: (C, e) = (80, 7) w = 36,
        // (112, 9) w = 51, (160, 15) w = 72, (208, 3) w = 102
#define DTW_REG_FIXED(CC, EE)                                                         \
    if (g.C == CC && g.e == EE) {                                                     \
        auto kern = k_dtw_reg<CC, P, EE>;                                            \
        kern<<<launch_detail::blocks_for(kern, warps), kDtwThreads, 0, s>>>(j, g.e, g.wl);           \
        return cudaGetLastError();                                                    \
    }
        DTW_REG_FIXED(80, 7) DTW_REG_FIXED(112, 9) DTW_REG_FIXED(160, 15) DTW_REG_FIXED(208, 3)
#undef DTW_REG_FIXED
#define DTW_REG_CASE(CC)                                                              \
    case CC: {                                                                        \
        auto kern = k_dtw_reg<CC, P, -1>;                                            \
        kern<<<launch_detail::blocks_for(kern, warps), kDtwThreads, 0, s>>>(j, g.e, g.wl);           \
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
        auto kern = k_dtw_wide<CC, P>;                                               \
        kern<<<launch_detail::blocks_for(kern, warps), kDtwThreads, 0, s>>>(j);                      \
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

// The row-phase thread-per-pair kernels for one launch of j.ph's rows:
// k_dtw_reg4p for bands of up to 64 slots, k_dtw_regp up to 208 (the
// register path only).
template <int P>
cudaError_t launch_dtw_phase_pt(const DtwJob &j, const DtwGeom &g, cudaStream_t s) {
    if (g.wide || g.C > kDtwRegMaxC) return cudaErrorInvalidValue;
    const int64_t warps = (j.npairs + 31) / 32;
    if (g.C > kDtwGroupMaxC) {
        // p = 1 and 2 only: the p = 4 and infinity variants of the widest
        // bands spill registers
        if constexpr (P == 1 || P == 2) {
#define DTW_REGP_CASE(CC)                                                                             \
    case CC: {                                                                                        \
        auto kern = k_dtw_regp<CC, P>;                                                               \
        kern<<<launch_detail::blocks_for(kern, warps), kDtwThreads, 0, s>>>(j, g.e, g.wl);            \
        return cudaGetLastError();                                                                    \
    }
            switch (g.C) {
                DTW_REGP_CASE(80) DTW_REGP_CASE(96) DTW_REGP_CASE(112) DTW_REGP_CASE(128)
                DTW_REGP_CASE(144) DTW_REGP_CASE(160) DTW_REGP_CASE(176) DTW_REGP_CASE(192)
                DTW_REGP_CASE(208)
                default: break;
            }
#undef DTW_REGP_CASE
        }
        return cudaErrorInvalidValue;
    }
    const bool xvec = (j.n % 4 == 0) && ((reinterpret_cast<uintptr_t>(j.db) & 15) == 0);
#define DTW_REG4P_FIXED(CC, EE)                                                                       \
    if (g.C == CC && g.e == EE) {                                                                     \
        auto kern = k_dtw_reg4p<CC, P, EE>;                                                          \
        kern<<<launch_detail::blocks_for(kern, warps), kDtwThreads, 0, s>>>(j, g.e, g.wl, xvec);      \
        return cudaGetLastError();                                                                    \
    }
    DTW_REG4P_FIXED(16, 3) DTW_REG4P_FIXED(32, 7) DTW_REG4P_FIXED(48, 11) DTW_REG4P_FIXED(64, 13)
#undef DTW_REG4P_FIXED
#define DTW_REG4P_CASE(CC)                                                                            \
    case CC: {                                                                                        \
        auto kern = k_dtw_reg4p<CC, P, -1>;                                                          \
        kern<<<launch_detail::blocks_for(kern, warps), kDtwThreads, 0, s>>>(j, g.e, g.wl, xvec);      \
        return cudaGetLastError();                                                                    \
    }
    switch (g.C) {
        DTW_REG4P_CASE(16) DTW_REG4P_CASE(32) DTW_REG4P_CASE(48) DTW_REG4P_CASE(64)
        default: return cudaErrorInvalidValue;
    }
#undef DTW_REG4P_CASE
}

}  // namespace dtwk

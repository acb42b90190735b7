// Band-constrained DTW_p with early abandoning (Sec. 4 recursion; early
// abandoning as cited in Sec. 3).  The paper's suffix recursion
//   q_{i,j} = |x_i - y_j|^p + min(q_{i+1,j}, q_{i,j+1}, q_{i+1,j+1})
// is evaluated here in the mirrored prefix form
//   D(i,j) = |x_i - y_j|^p + min(D(i-1,j), D(i,j-1), D(i-1,j-1)),
// D(-1,-1) = 0, other out-of-range or out-of-band cells +INF, which is the same
// minimum over the same warping paths.  Rows i = 0..n-1 are swept in order;
// a row holds the band cells j = i-w..i+w in "slots" k, column j = i - wl + k.
//
// Early abandoning: costs are >= 0 and fp32 addition of a non-negative term
// never decreases a value, so every path's fp32 sum is at least the minimum
// of any row it crosses; once a row minimum exceeds the threshold the final
// value does too, and the pair is abandoned (result +INF).
#pragma once
#include "common.cuh"

namespace dtwk {

constexpr int kDtwRegMaxC = 208;  // widest band kept in one thread's registers
constexpr int kDtwThreads = 128;
constexpr int kDtwGroupMaxC = 64;  // band widths processed 4 rows per window load
constexpr int kDtwPhaseRows = 64;  // rows per launch of the row-phase register kernel (a multiple of 8)

struct DtwGeom {
    int C;      // slots per pair (register path) or per warp (wide path)
    int e;      // bottom padding slots (register path), 0 for the wide path
    int wl;     // slot k holds column i - wl + k
    int padl;   // query copy left padding
    int ylen;   // query copy length
    bool wide;  // warp-split wide-band path
    int cl;     // wide path: slots per lane
};

inline DtwGeom dtw_geom(int n, int w) {
    DtwGeom g{};
    w = w < n - 1 ? w : n - 1;
    const int bw = 2 * w + 1;
    if (bw <= kDtwRegMaxC) {
        g.C = (bw + 15) / 16 * 16;
        g.e = g.C - bw;
        g.wl = w + g.e;
        g.wide = false;
        g.cl = 0;
    } else {
        int cl = 8;
        while (32 * cl < bw) cl *= 2;
        g.cl = cl;
        g.C = 32 * cl;
        g.e = 0;
        g.wl = w;
        g.wide = true;
    }
    // Register path: padl = wl puts row i's band window at padded index i, so
    // a group of 4 rows starting at a multiple of 4 reads one aligned span of
    // copy 0.  Wide path: padl = C (scalar loads).
    g.padl = g.wide ? g.C : g.wl;
    g.ylen = (n + g.padl + g.C + w + 8 + 3) / 4 * 4;
    return g;
}

// Warp path (dtw_lanes.cuh): G lanes per pair and CL slots per lane for the
// band 2w+1 (from the instantiated sets), or cl = 0 when the band needs more
// than 32 x 32 slots.  Groups of 32 give each pair the shortest chain of
// dependent steps (for launches of few pairs, where that latency sets the
// time); groups of 16, two per warp, halve the per-pair cost of the steps'
// bookkeeping (for launches of many pairs, where throughput does).
struct LanesShape {
    int g, cl;
};
inline LanesShape dtw_lanes_shape(int n, int w, bool many_pairs = false) {
    w = w < n - 1 ? w : n - 1;
    const int bw = 2 * w + 1;
    if (many_pairs && bw <= 16 * 32) {
        const int need = (bw + 15) / 16;
        const int set16[] = {4, 7, 10, 13, 16, 20, 26, 32};
        for (int c : set16)
            if (c >= need) return LanesShape{16, c};
    }
    const int need = (bw + 31) / 32;
    const int set32[] = {2, 3, 4, 5, 6, 7, 8, 10, 13, 16, 20, 24, 32};
    for (int c : set32)
        if (c >= need) return LanesShape{32, c};
    return LanesShape{0, 0};
}
inline int dtw_lanes_cl(int n, int w) { return dtw_lanes_shape(n, w).cl; }

cudaError_t launch_dtw_lanes_p1(const DtwJob &j, const DtwGeom &g, LanesShape ls, cudaStream_t s);
cudaError_t launch_dtw_lanes_p2(const DtwJob &j, const DtwGeom &g, LanesShape ls, cudaStream_t s);
cudaError_t launch_dtw_lanes_p4(const DtwJob &j, const DtwGeom &g, LanesShape ls, cudaStream_t s);
cudaError_t launch_dtw_lanes_pinf(const DtwJob &j, const DtwGeom &g, LanesShape ls, cudaStream_t s);

cudaError_t launch_dtw_p1(const DtwJob &j, const DtwGeom &g, cudaStream_t s);
cudaError_t launch_dtw_p2(const DtwJob &j, const DtwGeom &g, cudaStream_t s);
cudaError_t launch_dtw_p4(const DtwJob &j, const DtwGeom &g, cudaStream_t s);
cudaError_t launch_dtw_pinf(const DtwJob &j, const DtwGeom &g, cudaStream_t s);

cudaError_t launch_dtw_phase_p1(const DtwJob &j, const DtwGeom &g, cudaStream_t s);
cudaError_t launch_dtw_phase_p2(const DtwJob &j, const DtwGeom &g, cudaStream_t s);
cudaError_t launch_dtw_phase_p4(const DtwJob &j, const DtwGeom &g, cudaStream_t s);
cudaError_t launch_dtw_phase_pinf(const DtwJob &j, const DtwGeom &g, cudaStream_t s);

// One launch of the row-phase register kernel (j.ph), by the job's exponent.
inline cudaError_t launch_dtw_phase_by_p(const DtwJob &j, const DtwGeom &g, cudaStream_t s) {
    switch (j.p) {
        case 1: return launch_dtw_phase_p1(j, g, s);
        case 2: return launch_dtw_phase_p2(j, g, s);
        case 4: return launch_dtw_phase_p4(j, g, s);
        case 0: return launch_dtw_phase_pinf(j, g, s);
        default: return cudaErrorInvalidValue;
    }
}

// DTW of a job by its exponent j.p (1, 2, 4, or 0 for p = infinity).
inline cudaError_t launch_dtw_by_p(const DtwJob &j, const DtwGeom &g, cudaStream_t s) {
    switch (j.p) {
        case 1: return launch_dtw_p1(j, g, s);
        case 2: return launch_dtw_p2(j, g, s);
        case 4: return launch_dtw_p4(j, g, s);
        case 0: return launch_dtw_pinf(j, g, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dtwk

// Warp path of the band DTW in a one-row-per-step wavefront (Sec. 4
// recursion): a group of G lanes (16 or 32) steps one pair; lane l owns the
// band slots l*CL .. l*CL+CL-1 (slot k of row i holds column i - wl + k) and,
// at step s of the pair, computes its slots of row s - l.  Cell (i, k) needs
// (i-1, k) and (i-1, k+1) from the previous row and (i, k-1) from its own:
//  - the lane's first cell needs the last slot of row i on lane l-1, which
//    computed row i one step earlier (a shuffle at the start of the step);
//  - the lane's last cell needs slot (l+1)*CL of row i-1, which lane l+1
//    computes as its FIRST cell of the same step: it is shuffled down right
//    after the first cells and used CL-1 cells later.
// So every lane computes a row segment at every step, with one pair per
// group and no idle steps, where a two-steps-per-row wavefront (dtw_lanes.cuh)
// needs a second pair to fill its gaps.  Lanes switch to the group's next pair
// one step apart (lane l at the pair's start step + l), so the stagger, and
// the neighbours' values each lane reads, carry over from pair to pair; a
// lane at row 0 takes the row -1 values (D(-1,-1) = 0) instead of its right
// neighbour's.
//
// The band's 2w+1 slots are the top of the G*CL slots; the E slots below
// them are padding (compile-time).  Lanes whose slots all lie in the padding
// step nothing; in the lane that holds the band's lowest slot, the padding
// slots' window values are +INF, so their cells are +INF (|x - INF| + m) and
// never feed the band: one register per row is reset as the window slides.  Pairs start at block boundaries (every CL steps, one
// compile-time rotation of the window registers per step).
//
// Each lane's next two rows' x values and new window values are in flight
// while it computes the current one (one row ahead left the loads exposed).
//
// Abandoning: after each block, the group's wavefront (each lane's last row
// of the current pair; the row -1 values for lanes that have not reached it)
// is a cut that every warping path crosses: within a row a path moves to
// higher slots, and from row to row to the same or a lower slot, while lane
// l + 1 (higher slots) is one row behind lane l.  Its minimum bounds DTW^p.
#pragma once
#include "dtw_kernels.cuh"

namespace dtwk {

template <int CL, int G, int P, int E>
__global__ void __launch_bounds__(kDtwThreads, 4) k_dtw_wave(DtwJob j) {
    static_assert(G == 16 || G == 32, "lane groups of 16 or 32");
    static_assert(CL >= 2 && CL <= 16 && E >= 0 && E < G * CL, "2 to 16 slots per lane");
    constexpr int kPadLanes = E / CL;  // lanes below this hold only padding
    constexpr int kPadCells = E % CL;  // cells of lane kPadLanes below the band
    constexpr int kIdle = 1 << 30;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int gbase = lane & ~(G - 1);
    const unsigned gmask = G == 32 ? 0xffffffffu : (0xffffu << gbase);
    const int n = j.n;
    const int w = min(j.w, n - 1);
    const int wl = w + E;  // the host checks 2w + 1 + E == G * CL
    const int k0 = gl * CL;
    const bool pad_lane = gl < kPadLanes;
    const bool part_lane = gl == kPadLanes;
    const int lane_diag = wl / CL, c_diag = wl % CL;
    // row -1: D(-1, -1) = 0 at slot wl; the value lane l's last cell reads
    // above it at row 0 is slot k0 + CL of row -1
    const float init_up = (k0 + CL == wl) ? 0.0f : kInf;
    const int64_t qstride = (int64_t)4 * j.qc.ylen;
    if (j.npairs_dev) j.npairs = (int64_t)*j.npairs_dev;
    unsigned long long n_skip = 0, n_comp = 0, n_aband = 0, n_rows = 0, n_cells = 0;

    float D[CL], yw[CL];
#pragma unroll
    for (int u = 0; u < CL; ++u) {
        D[u] = kInf;
        yw[u] = 0.0f;
    }
    float last = kInf;         // this lane's last slot of its latest row (for lane l + 1)
    float nx = 0.0f, ny = 0.0f;    // the next row's x value and new window value
    float nx2 = 0.0f, ny2 = 0.0f;  // the row after it
    const float *xr = j.db, *yr = j.qc.data;  // the pair this lane steps
    int64_t mpi = -1;                          // its pair index
    int T = kIdle;                             // the step of its row 0
    int64_t dead = -1;                         // the last pair the group abandoned

    // the group's current pair (uniform in the group)
    bool g_act = false;
    int64_t g_pi = -1;
    int g_q = 0, g_c = 0, g_T0 = 0;

    // Pairs come `chunk` at a time from the cursor; each lane checks one of
    // the chunk against the threshold, and a ballot keeps the rest.
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x >> 5) * (32 / G);
    const int64_t per = j.npairs / (2 * groups);
    const int chunk = per < 1 ? 1 : (per > G ? G : (int)per);
    int64_t cbase = 0;
    unsigned cmask = 0;
    int my_q = 0, my_c = 0;
    float my_lbi = 0.0f;
    bool exhausted = false;

    // The group's next pair, started at step t0 (lane l's row 0 at t0 + l).
    auto fetch = [&](int t0) {
        g_act = false;
        while (!exhausted) {
            while (cmask == 0) {
                unsigned long long ch = 0;
                if (gl == 0) ch = atomicAdd(j.cursor, 1ull);
                ch = __shfl_sync(gmask, ch, gbase);
                cbase = (int64_t)ch * chunk;
                if (cbase >= j.npairs) {
                    exhausted = true;
                    break;
                }
                const int64_t pi = cbase + gl;
                bool valid;
                fetch_pair(j, pi, my_q, my_c, valid);
                valid = valid && gl < chunk;
                my_lbi = 0.0f;
                if (valid && j.pair_lbi) {
                    my_lbi = j.pair_lbi[pi];
                    const float thr = j.bsf ? load_threshold(j.bsf + my_q) : j.fixed_thr;
                    if (my_lbi > thr * (1.0f + j.slack)) {
                        j.res[pi] = kInf;
                        ++n_skip;
                        valid = false;
                    }
                }
                cmask = __ballot_sync(gmask, valid) >> gbase;
            }
            if (exhausted) break;
            const int src = __ffs(cmask) - 1;
            cmask &= cmask - 1;
            const int q = __shfl_sync(gmask, my_q, gbase + src);
            const int c = __shfl_sync(gmask, my_c, gbase + src);
            const float lbi = __shfl_sync(gmask, my_lbi, gbase + src);
            const int64_t pi = cbase + src;
            if (j.pair_lbi) {
                // the threshold may have fallen since the chunk was checked
                float thr = j.bsf ? load_threshold(j.bsf + q) : j.fixed_thr;
                thr = __shfl_sync(gmask, thr, gbase);
                if (lbi > thr * (1.0f + j.slack)) {
                    if (gl == 0) {
                        j.res[pi] = kInf;
                        ++n_skip;
                    }
                    continue;
                }
            }
            g_act = true;
            g_pi = pi;
            g_q = q;
            g_c = c;
            g_T0 = t0;
            if (gl == 0) ++n_comp;
            break;
        }
    };

    int t = 0;
    fetch(0);
    int t_end = g_act ? kIdle : 0;  // once no pair is left: the step after the last lane's last row
    // the steps shuffle across the whole warp, so the warp steps while either
    // of its groups has rows left
    while (__any_sync(0xffffffffu, t < t_end)) {
        // one block of CL steps; step R uses window rotation R
        const int t_switch = g_act ? g_T0 + gl : -1;  // the step this lane starts the group's pair
#define WAVE_STEP(R)                                                                                          \
    {                                                                                                         \
        const int ts = t + (R);                                                                               \
        if (ts == t_switch) {                                                                                 \
            /* this lane starts the group's current pair: row -1 values, the window of row 0 */              \
            xr = j.db + (int64_t)g_c * n;                                                                     \
            yr = j.qc.data + (int64_t)g_q * qstride + j.qc.padl;                                              \
            mpi = g_pi;                                                                                       \
            T = ts;                                                                                           \
            _Pragma("unroll") for (int u = 0; u < CL; ++u) D[u] = (k0 + u == wl) ? 0.0f : kInf;             \
            _Pragma("unroll") for (int u = 0; u < CL - 1; ++u)                                                \
                yw[(u + (R)) % CL] = (u < kPadCells && part_lane) ? kInf : __ldg(yr + (k0 + u - wl));         \
            nx = __ldg(xr);                                                                                   \
            ny = __ldg(yr + (k0 + CL - 1 - wl));                                                              \
            if (n > 1) {                                                                                      \
                nx2 = __ldg(xr + 1);                                                                          \
                ny2 = __ldg(yr + (1 + k0 + CL - 1 - wl));                                                     \
            }                                                                                                 \
        }                                                                                                     \
        const int r = ts - T;                                                                                 \
        const bool due = !pad_lane && (unsigned)r < (unsigned)n;                                              \
        float left = __shfl_up_sync(gmask, last, 1, G);                                                       \
        if (gl == 0) left = kInf;                                                                             \
        float xi = 0.0f;                                                                                      \
        if (due) {                                                                                            \
            yw[(CL - 1 + (R)) % CL] = ny;                                                                     \
            /* the padding slot just below the band: a +INF window value makes its cells +INF */             \
            if (kPadCells > 0 && part_lane) yw[(kPadCells - 1 + (R)) % CL] = kInf;                            \
            xi = nx;                                                                                          \
            nx = nx2;                                                                                         \
            ny = ny2;                                                                                         \
            if (r + 2 < n) {                                                                                  \
                nx2 = __ldg(xr + r + 2);                                                                      \
                ny2 = __ldg(yr + (r + 2 - wl + k0 + CL - 1));                                                 \
            }                                                                                                 \
            const float c0 = dtw_cost<P>(xi - yw[(R) % CL], min3f(D[0], D[1], left));                       \
            D[0] = c0;                                                                                        \
        }                                                                                                     \
        float up = __shfl_down_sync(gmask, D[0], 1, G);                                                       \
        if (gl == G - 1) up = kInf;                                                                           \
        if (r == 0) up = init_up;                                                                             \
        if (due) {                                                                                            \
            _Pragma("unroll") for (int u = 1; u < CL; ++u) {                                                  \
                const float above = (u + 1 < CL) ? D[(u + 1 < CL) ? u + 1 : u] : up;                          \
                const float v = dtw_cost<P>(xi - yw[(u + (R)) % CL], min3f(D[u], above, D[u - 1]));          \
                D[u] = v;                                                                                     \
            }                                                                                                 \
            last = D[CL - 1];                                                                                 \
            if (r == n - 1 && gl == lane_diag && mpi != dead) {                                               \
                /* the pair's DTW^p: slot wl of row n - 1 */                                                  \
                float val = kInf;                                                                             \
                _Pragma("unroll") for (int u = 0; u < CL; ++u) val = (u == c_diag) ? D[u] : val;             \
                int q, c;                                                                                     \
                bool valid;                                                                                   \
                fetch_pair(j, mpi, q, c, valid);                                                              \
                n_rows += (unsigned long long)n;                                                              \
                n_cells += (unsigned long long)band_cells(n, n, w);                                           \
                if (!j.bsf && val > j.fixed_thr) val = kInf;                                                  \
                j.res[mpi] = j.root_out ? root_p(val, P) : val;                                               \
                if (j.bsf) update_threshold(j.bsf, j.gmin, j.k, q, c % j.k, val);                             \
            }                                                                                                 \
        }                                                                                                     \
    }
        WAVE_STEP(0)
        if constexpr (CL > 1) WAVE_STEP(1)
        if constexpr (CL > 2) WAVE_STEP(2)
        if constexpr (CL > 3) WAVE_STEP(3)
        if constexpr (CL > 4) WAVE_STEP(4)
        if constexpr (CL > 5) WAVE_STEP(5)
        if constexpr (CL > 6) WAVE_STEP(6)
        if constexpr (CL > 7) WAVE_STEP(7)
        if constexpr (CL > 8) WAVE_STEP(8)
        if constexpr (CL > 9) WAVE_STEP(9)
        if constexpr (CL > 10) WAVE_STEP(10)
        if constexpr (CL > 11) WAVE_STEP(11)
        if constexpr (CL > 12) WAVE_STEP(12)
        if constexpr (CL > 13) WAVE_STEP(13)
        if constexpr (CL > 14) WAVE_STEP(14)
        if constexpr (CL > 15) WAVE_STEP(15)
#undef WAVE_STEP
        t += CL;
        if (!g_act) continue;
        // lane 0 has passed row n - 1 of the current pair: the next one starts
        bool next = t >= g_T0 + n;
        bool abandoned = false;
        if (!next && j.abandon) {
            // the wavefront of the current pair: each lane's last row of it,
            // or the row -1 values where the lane has not started it
            float mn;
            if (pad_lane) {
                mn = kInf;
            } else if (mpi == g_pi && t > T) {
                mn = D[0];
#pragma unroll
                for (int u = 1; u < CL; ++u) mn = fminf(mn, D[u]);
            } else {
                mn = (k0 <= wl && wl < k0 + CL) ? 0.0f : kInf;
            }
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(gmask, mn, o));
            float thr = j.bsf ? load_threshold(j.bsf + g_q) : j.fixed_thr;
            thr = __shfl_sync(gmask, thr, gbase);
            if (mn > thr) {
                dead = g_pi;
                if (gl == 0) {
                    ++n_aband;
                    // rows every lane of the group has passed
                    const int rows = max(0, min(n, t - g_T0 - (G - 1)));
                    n_rows += (unsigned long long)rows;
                    n_cells += (unsigned long long)band_cells(rows, n, w);
                    j.res[g_pi] = kInf;
                }
                next = true;
                abandoned = true;
            }
        }
        if (next) {
            fetch(t);
            // with no pair left: after an abandon nothing remains to step;
            // after a completion, the lanes up to the result's lane finish
            if (!g_act) t_end = abandoned ? t : g_T0 + n + G;
        }
    }
    if (j.counters) {
        n_skip = __reduce_add_sync(0xffffffffu, (unsigned)n_skip);
        n_comp = __reduce_add_sync(0xffffffffu, (unsigned)n_comp);
        n_aband = __reduce_add_sync(0xffffffffu, (unsigned)n_aband);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            n_rows += __shfl_xor_sync(0xffffffffu, n_rows, o);
            n_cells += __shfl_xor_sync(0xffffffffu, n_cells, o);
        }
        if (lane == 0) {
            if (n_skip) atomicAdd(j.counters + CNT_DTW_SKIP, n_skip);
            if (n_comp) atomicAdd(j.counters + CNT_DTW_COMPUTED, n_comp);
            if (n_aband) atomicAdd(j.counters + CNT_DTW_ABANDONED, n_aband);
            if (n_rows) atomicAdd(j.counters + CNT_DTW_ROWS, n_rows);
            if (n_cells) atomicAdd(j.counters + CNT_DTW_CELLS, n_cells);
        }
    }
}

}  // namespace dtwk

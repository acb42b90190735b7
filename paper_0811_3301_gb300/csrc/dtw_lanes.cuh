// Warp path of the band DTW (Sec. 4 recursion, prefix form as in dtw.cuh):
// a group of G lanes (16 or 32) shares the band of a pair, and each group
// keeps two pairs in flight.  Used for bands too wide for one thread's registers and
// for long series when there are too few pairs to fill the GPU one thread
// per pair (the latency of one long DTW then sets the stage time).
//
// Lane l of a group owns the band slots l*CL .. l*CL+CL-1; slot k of row i
// holds column i - w + k.  Cell (i, k) needs (i-1, k) and (i-1, k+1) from the previous
// row and (i, k-1) from its own row, so lane l can compute row i one step
// after lane l-1 computed row i and lane l+1 computed row i-1.  A pair whose
// rows start at step T0 therefore has lane l compute its row i at step
// T0 + l + 2i, and each lane would idle every other step; the second pair,
// started at a step of the other parity, fills those steps.  At even steps
// every lane works on its register set X and at odd steps on set Y (set X of
// lane l belongs to pair slot l & 1), so the steps never diverge; only the
// completions and restarts of a group's pairs, between blocks of steps, do.
// Two groups of 16 lanes per warp halve the per-pair cost of the steps'
// bookkeeping against one group of 32 with half the slots per lane.
//
// The query window of a lane slides by one column per row.  Its registers
// are addressed through a rotation that is a compile-time constant in each of
// CL unrolled rows, so the slide costs one load and no register moves.
//
// Abandoning: costs are >= 0 and fp32 addition of a non-negative term never
// decreases a value, so a path's fp32 sum is at least the value of any cell
// it passes.  Every path from (0,0) to (n-1,n-1) leaves the cells computed so
// far through a cell of the wavefront (the last row each lane computed; the
// row -1 initial values, with D(-1,-1) = 0, on lanes that have not started),
// so the wavefront minimum bounds DTW^p from below, and the pair is abandoned
// once that minimum exceeds the threshold.
#pragma once
#include "dtw_kernels.cuh"

namespace dtwk {

// D[c] = +INF for a runtime c in [1, CL): a jump to one store, taken by one lane.
template <int CL>
__device__ __forceinline__ void lanes_kill(float (&D)[CL], int c) {
    switch (c) {
#define LANES_KILL(U)                          \
    case U:                                    \
        if constexpr (U < CL) D[U] = kInf;     \
        break;
        LANES_KILL(1) LANES_KILL(2) LANES_KILL(3) LANES_KILL(4) LANES_KILL(5) LANES_KILL(6) LANES_KILL(7)
        LANES_KILL(8) LANES_KILL(9) LANES_KILL(10) LANES_KILL(11) LANES_KILL(12) LANES_KILL(13) LANES_KILL(14)
        LANES_KILL(15) LANES_KILL(16) LANES_KILL(17) LANES_KILL(18) LANES_KILL(19) LANES_KILL(20) LANES_KILL(21)
        LANES_KILL(22) LANES_KILL(23) LANES_KILL(24) LANES_KILL(25) LANES_KILL(26) LANES_KILL(27) LANES_KILL(28)
        LANES_KILL(29) LANES_KILL(30) LANES_KILL(31)
#undef LANES_KILL
        default: break;
    }
}

// One step of one register set: the set's pair computes its next row on this
// lane if the row is due.  R: rotation of the window registers for this row.
// nx, ny: the next row's x value and new window value, loaded one row ahead
// (the set's next row comes two steps later) so that no step waits on them.
template <int CL, int G, int P, int R>
__device__ __forceinline__ void lanes_step(float (&D)[CL], float (&yw)[CL], float &nx, float &ny,
                                           const float *__restrict__ x, const float *__restrict__ yq, int s0, int t,
                                           int n, int w, int k0, bool computes, bool reset_dead, int c_dead,
                                           int gl, float &pub_first, float &pub_last) {
    float left = __shfl_up_sync(0xffffffffu, pub_last, 1, G);
    float up = __shfl_down_sync(0xffffffffu, pub_first, 1, G);
    if (gl == 0) left = kInf;
    if (gl == G - 1) up = kInf;
    const int d = t - s0;  // even whenever this set's pair is due on this lane
    if (computes && d >= 0 && d < 2 * n) {
        const int i = d >> 1;
        float xi;
        if (i == 0) {
#pragma unroll
            for (int u = 0; u < CL; ++u) yw[(u + R) % CL] = __ldg(yq + (k0 + u - w));
            xi = __ldg(x);
        } else {
            yw[(CL - 1 + R) % CL] = ny;
            xi = nx;
        }
        if (i + 1 < n) {
            nx = __ldg(x + i + 1);
            ny = __ldg(yq + (i + 1 - w + k0 + CL - 1));
        }
#pragma unroll
        for (int u = 0; u < CL; ++u) {
            const float above = (u + 1 < CL) ? D[(u + 1 < CL) ? u + 1 : u] : up;
            const float below = (u > 0) ? D[(u > 0) ? u - 1 : 0] : left;
            const float m = min3f(D[u], above, below);
            const float df = xi - yw[(u + R) % CL];
            D[u] = dtw_cost<P>(df, m);
        }
        if (reset_dead) lanes_kill<CL>(D, c_dead);  // slot 2w+1 (outside the band) reads +INF next row
    }
    pub_first = D[0];
    pub_last = D[CL - 1];
}

// CL consecutive step pairs (X at even t, Y at odd t), one rotation each.
template <int CL, int G, int P, int R>
__device__ __forceinline__ void lanes_block(float (&DX)[CL], float (&DY)[CL], float (&yX)[CL], float (&yY)[CL],
                                            float (&nxt)[4], const float *xX, const float *xY, const float *qX,
                                            const float *qY, int sX, int sY, int t, int n, int w, int k0,
                                            bool computes, bool reset_dead, int c_dead, int gl, float &pub_first,
                                            float &pub_last) {
    if constexpr (R < CL) {
        lanes_step<CL, G, P, R>(DX, yX, nxt[0], nxt[1], xX, qX, sX, t, n, w, k0, computes, reset_dead, c_dead, gl,
                                pub_first, pub_last);
        lanes_step<CL, G, P, R>(DY, yY, nxt[2], nxt[3], xY, qY, sY, t + 1, n, w, k0, computes, reset_dead, c_dead,
                                gl, pub_first, pub_last);
        lanes_block<CL, G, P, R + 1>(DX, DY, yX, yY, nxt, xX, xY, qX, qY, sX, sY, t + 2, n, w, k0, computes,
                                     reset_dead, c_dead, gl, pub_first, pub_last);
    }
}

// Register budget: the steps are chains of dependent cells, so the kernel
// lives on the number of warps in flight.  Up to 13 slots per lane fit 128
// registers (16 warps per SM) and up to 20 fit 168 (12 warps) without
// spilling; wider lanes keep what they need.
template <int CL, int G, int P>
__global__ void __launch_bounds__(kDtwThreads, (CL <= 13 ? 4 : (CL <= 20 ? 3 : 1))) k_dtw_lanes(DtwJob j) {
    static_assert(G == 16 || G == 32, "lane groups of 16 or 32");
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);      // lane within the group
    const int gbase = lane & ~(G - 1);  // first lane of the group
    const unsigned gmask = G == 32 ? 0xffffffffu : (0xffffu << gbase);
    const int n = j.n;
    const int w = min(j.w, n - 1);
    const int top = 2 * w;                 // highest band slot; 2w+1 <= G*CL
    const int lane_top = top / CL;
    const int c_dead = (top + 1) % CL;     // slot 2w+1 lies in lane_top when c_dead > 0
    const bool reset_dead = (gl == lane_top) && c_dead > 0;
    const int lane_diag = w / CL, c_diag = w % CL;
    const int k0 = gl * CL;
    const bool computes = gl <= lane_top;
    const int64_t qstride = (int64_t)4 * j.qc.ylen;
    constexpr int kIdle = 1 << 30;
    if (j.npairs_dev) j.npairs = (int64_t)*j.npairs_dev;
    unsigned long long n_skip = 0, n_comp = 0, n_aband = 0, n_rows = 0, n_cells = 0;

    float DX[CL], DY[CL], yX[CL], yY[CL];
    float nxt[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // next-row x and window values of sets X and Y
#pragma unroll
    for (int u = 0; u < CL; ++u) {
        DX[u] = kInf;
        DY[u] = kInf;
        yX[u] = 0.0f;
        yY[u] = 0.0f;
    }
    const float *xX = j.db, *xY = j.db, *qX = j.qc.data, *qY = j.qc.data;
    int sX = kIdle, sY = kIdle;  // step of this lane's row 0 of the set's pair
    // pair slots (uniform within the group)
    bool act[2] = {false, false};
    int64_t spi[2] = {0, 0};
    int sq[2] = {0, 0}, sc[2] = {0, 0}, T0[2] = {0, 0};
    float pub_first = kInf, pub_last = kInf;

    // Pairs are taken `chunk` at a time from the cursor: each lane of the group
    // loads one pair of the chunk and drops it if its bound already exceeds
    // the threshold, and a ballot keeps the rest in a group-uniform queue.
    // Long lists of mostly skipped pairs take G per fetch; short lists take
    // fewer, so that every group gets pairs.
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x >> 5) * (32 / G);
    int64_t per = j.npairs / (2 * groups);
    const int chunk = per < 1 ? 1 : (per > G ? G : (int)per);
    int64_t cbase = 0;
    unsigned cmask = 0;
    int my_q = 0, my_c = 0;
    float my_lbi = 0.0f;
    auto refill = [&]() -> bool {
        while (cmask == 0) {
            unsigned long long ch = 0;
            if (gl == 0) ch = atomicAdd(j.cursor, 1ull);
            ch = __shfl_sync(gmask, ch, gbase);
            cbase = (int64_t)ch * chunk;
            if (cbase >= j.npairs) return false;
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
        return true;
    };

    // Takes the next pair for slot ps, with rows starting at step t0 (t0 has
    // the parity of ps).
    auto start = [&](int ps, int t0) {
        act[ps] = false;
        while (refill()) {
            const int src = __ffs(cmask) - 1;
            cmask &= cmask - 1;
            const int q = __shfl_sync(gmask, my_q, gbase + src);
            const int c = __shfl_sync(gmask, my_c, gbase + src);
            const float lbi = __shfl_sync(gmask, my_lbi, gbase + src);
            const int64_t pi = cbase + src;
            if (j.pair_lbi) {
                // the threshold may have dropped since the chunk was loaded
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
            act[ps] = true;
            spi[ps] = pi;
            sq[ps] = q;
            sc[ps] = c;
            T0[ps] = t0;
            if (gl == 0) ++n_comp;
            break;
        }
        const bool mine_x = (gl & 1) == ps;
        const float *xr = j.db + (int64_t)sc[ps] * n;
        const float *qr = j.qc.data + (int64_t)sq[ps] * qstride + j.qc.padl;
        const int s0 = act[ps] ? t0 + gl : kIdle;
        if (mine_x) {
            xX = xr;
            qX = qr;
            sX = s0;
#pragma unroll
            for (int u = 0; u < CL; ++u) DX[u] = (k0 + u == w) ? 0.0f : kInf;
        } else {
            xY = xr;
            qY = qr;
            sY = s0;
#pragma unroll
            for (int u = 0; u < CL; ++u) DY[u] = (k0 + u == w) ? 0.0f : kInf;
        }
    };

    int t = 0;
    start(0, 0);
    start(1, 1);
    // the steps shuffle across the whole warp, so the warp keeps stepping
    // while either of its groups has a pair
    while (__any_sync(0xffffffffu, act[0] || act[1])) {
        // t is even here
        lanes_block<CL, G, P, 0>(DX, DY, yX, yY, nxt, xX, xY, qX, qY, sX, sY, t, n, w, k0, computes, reset_dead,
                                 c_dead, gl, pub_first, pub_last);
        t += 2 * CL;
        // completions and abandons of the group's two slots (t is the next step)
#pragma unroll
        for (int ps = 0; ps < 2; ++ps) {
            if (!act[ps]) continue;
            const bool mine_x = (gl & 1) == ps;
            // lane_diag computes the last row at T0 + lane_diag + 2(n-1)
            const bool done = t > T0[ps] + lane_diag + 2 * (n - 1);
            bool ab = false;
            float val = kInf;
            if (done) {
                float v = kInf;
#pragma unroll
                for (int u = 0; u < CL; ++u) v = sel_eq(u, c_diag, mine_x ? DX[u] : DY[u], v);
                val = __shfl_sync(gmask, v, gbase + lane_diag);
            } else if (j.abandon) {
                float mn = kInf;
#pragma unroll
                for (int u = 0; u < CL; ++u) {
                    const float dv = mine_x ? DX[u] : DY[u];
                    mn = fminf(mn, (k0 + u <= top) ? dv : kInf);
                }
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(gmask, mn, o));
                float thr = j.bsf ? load_threshold(j.bsf + sq[ps]) : j.fixed_thr;
                thr = __shfl_sync(gmask, thr, gbase);
                ab = mn > thr;
            }
            if (done || ab) {
                if (gl == 0) {
                    if (ab) {
                        ++n_aband;
                        const int rows = max(0, min(n, (t - T0[ps] - lane_top) / 2));
                        n_rows += (unsigned long long)rows;
                        n_cells += (unsigned long long)band_cells(rows, n, w);
                        val = kInf;
                    } else {
                        n_rows += (unsigned long long)n;
                        n_cells += (unsigned long long)band_cells(n, n, w);
                    }
                    if (!j.bsf && val > j.fixed_thr) val = kInf;
                    j.res[spi[ps]] = j.root_out ? root_p(val, P) : val;
                    if (!ab && j.bsf) update_threshold(j.bsf, j.gmin, j.k, sq[ps], sc[ps] % j.k, val);
                }
                start(ps, t + ps);
            }
        }
        // the next (even) step reads what the neighbours' Y sets hold now,
        // including the initial values of a pair just started
        pub_first = DY[0];
        pub_last = DY[CL - 1];
    }
    if (j.counters) {
        n_skip = __reduce_add_sync(0xffffffffu, (unsigned)n_skip);
        if (lane == 0 && n_skip) atomicAdd(j.counters + CNT_DTW_SKIP, n_skip);
        if (gl == 0) {
            if (n_rows) atomicAdd(j.counters + CNT_DTW_ROWS, n_rows);
            if (n_cells) atomicAdd(j.counters + CNT_DTW_CELLS, n_cells);
            if (n_comp) atomicAdd(j.counters + CNT_DTW_COMPUTED, n_comp);
            if (n_aband) atomicAdd(j.counters + CNT_DTW_ABANDONED, n_aband);
        }
    }
}

}  // namespace dtwk

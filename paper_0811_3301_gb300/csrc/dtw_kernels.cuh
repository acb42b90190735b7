// DTW kernel bodies, instantiated per band width in dtw_p1.cu / dtw_p2.cu.
#pragma once
#include "dtw.cuh"

namespace dtwk {

// Update the k-NN thresholds of query q after a completed DTW value d
// (power space) of candidate c: group minima gmin[q][g] (g = c mod k) and the
// bound bsf[q] = max_g gmin[q][g], an upper bound on the k-th best distance
// because the k groups hold k distinct candidates.  Both only decrease.
__device__ __forceinline__ void update_threshold(uint32_t *bsf, uint32_t *gmin, int k, int q, int g,
                                                 float d) {
    const uint32_t bits = __float_as_uint(d);
    if (k == 1) {
        atomicMin(bsf + q, bits);
        return;
    }
    uint32_t old = atomicMin(gmin + (int64_t)q * k + g, bits);
    if (bits < old) {
        uint32_t mx = 0;
        for (int t = 0; t < k; ++t) {
            uint32_t v = *(volatile uint32_t *)(gmin + (int64_t)q * k + t);
            mx = v > mx ? v : mx;
        }
        atomicMin(bsf + q, mx);
    }
}

__device__ __forceinline__ void fetch_pair(const DtwJob &j, int64_t pi, int &q, int &c, bool &valid) {
    valid = pi < j.npairs;
    q = 0;
    c = 0;
    if (valid) {
        if (j.pairs) {
            Pair pr = j.pairs[pi];
            q = pr.q;
            c = pr.c;
        } else {
            c = (int)pi;
            q = j.per_pair_y ? (int)pi : 0;
        }
        if (c < 0) valid = false;
    }
}

// One band cell: slot K of the current row.  D[K] holds D(i-1, j-1) on entry,
// D[K+1] holds D(i-1, j), D[K-1] already holds D(i, j-1).
template <int K, int C, int P>
__device__ __forceinline__ void dtw_cell(float (&D)[C], float xi, float yv) {
    float above, below;
    if constexpr (K + 1 < C) above = D[K + 1]; else above = kInf;
    if constexpr (K > 0) below = D[K - 1]; else below = kInf;
    const float m = min3f(D[K], above, below);
    const float d = xi - yv;
    D[K] = dtw_cost<P>(d, m);
}
#define DTW_CELL(K, YV) dtw_cell<K, C, P>(D, xi, YV);

// One band cell given its difference d = x_i - y_j.
template <int K, int C, int P>
__device__ __forceinline__ void dtw_cell_d(float (&D)[C], float d) {
    float above, below;
    if constexpr (K + 1 < C) above = D[K + 1]; else above = kInf;
    if constexpr (K > 0) below = D[K - 1]; else below = kInf;
    D[K] = dtw_cost<P>(d, min3f(D[K], above, below));
}

// Differences x - y of two adjacent slots by one packed fp32x2 fma (y * -1 +
// x: the same rounding as x - y).  They are off the row's dependency chain,
// which runs through the minimum and the cost.
__device__ __forceinline__ float2 dtw_diff2(float xi, float ya, float yb) {
    return __ffma2_rn(make_float2(ya, yb), make_float2(-1.0f, -1.0f), make_float2(xi, xi));
}

// Cells K..C-1, four per 128-bit load of the query window.
template <int K, int C, int P>
__device__ __forceinline__ void dtw_cells_from(float (&D)[C], float xi, const float4 *yb) {
    if constexpr (K < C) {
        // (packed differences here measured slower: this kernel holds up to
        // 255 registers already)
        const float4 t = __ldg(yb + (K >> 2));
        dtw_cell<K, C, P>(D, xi, t.x);
        dtw_cell<K + 1, C, P>(D, xi, t.y);
        dtw_cell<K + 2, C, P>(D, xi, t.z);
        dtw_cell<K + 3, C, P>(D, xi, t.w);
        dtw_cells_from<K + 4, C, P>(D, xi, yb);
    }
}

// One row i of the register path: the band window of the query read from
// the shifted copy that puts column i - wl on a 16-byte boundary, the row
// entered at slot e (a jump on the uniform e).
template <int C, int P>
__device__ __forceinline__ void reg_row(float (&D)[C], float xi, const float *__restrict__ yc, int i, int e, int wl,
                                        int padl, int ylen) {
    const int a = i - wl + padl;
    const int r = a & 3;
    const float4 *yb = reinterpret_cast<const float4 *>(yc + r * ylen + (a - r));
    const float4 h0 = __ldg(yb + 0), h1 = __ldg(yb + 1), h2 = __ldg(yb + 2), h3 = __ldg(yb + 3);
    switch (e) {
        case 0: DTW_CELL(0, h0.x) [[fallthrough]];
        case 1: DTW_CELL(1, h0.y) [[fallthrough]];
        case 2: DTW_CELL(2, h0.z) [[fallthrough]];
        case 3: DTW_CELL(3, h0.w) [[fallthrough]];
        case 4: DTW_CELL(4, h1.x) [[fallthrough]];
        case 5: DTW_CELL(5, h1.y) [[fallthrough]];
        case 6: DTW_CELL(6, h1.z) [[fallthrough]];
        case 7: DTW_CELL(7, h1.w) [[fallthrough]];
        case 8: DTW_CELL(8, h2.x) [[fallthrough]];
        case 9: DTW_CELL(9, h2.y) [[fallthrough]];
        case 10: DTW_CELL(10, h2.z) [[fallthrough]];
        case 11: DTW_CELL(11, h2.w) [[fallthrough]];
        case 12: DTW_CELL(12, h3.x) [[fallthrough]];
        case 13: DTW_CELL(13, h3.y) [[fallthrough]];
        case 14: DTW_CELL(14, h3.z) [[fallthrough]];
        default: DTW_CELL(15, h3.w)
    }
    dtw_cells_from<16, C, P>(D, xi, yb);
}

__device__ __forceinline__ float f4_at(const float4 &v, int c) {
    return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

// Rows i and i + 1 of the register path for a compile-time bottom padding E,
// skewed by one slot: row i's slot K + 1 and row i + 1's slot K are the same
// column, so one query value serves both, and the two rows' chains (each cell
// waits on the one below it) run side by side instead of one after the
// other.  Each cell takes the operands of the one-row order, so the values
// are bit-identical to two calls of reg_row.  Reads the query window of row
// i up to slot C + 3 (row i + 1's last slot and the rest of its 16-byte
// piece), which the copies' right padding holds.
template <int C, int P, int E>
__device__ __forceinline__ void reg_rows2(float (&D)[C], float x0, float x1, const float *__restrict__ yc, int i,
                                          int wl, int padl, int ylen) {
    static_assert(E >= 0 && E < 16 && C % 16 == 0, "bottom padding below 16, C a multiple of 16");
    const int a = i - wl + padl;
    const int r = a & 3;
    const float4 *yb = reinterpret_cast<const float4 *>(yc + r * ylen + (a - r));
    float4 ch = __ldg(yb + (E >> 2));
    float a_k = dtw_cost<P>(x0 - f4_at(ch, E & 3), min3f(D[E], (E + 1 < C) ? D[(E + 1 < C) ? E + 1 : E] : kInf, kInf));
    float b_prev = kInf;
#pragma unroll
    for (int K = E; K < C; ++K) {
        if (((K + 1) & 3) == 0) ch = __ldg(yb + ((K + 1) >> 2));
        const float yv = f4_at(ch, (K + 1) & 3);
        float a_next = kInf;
        if (K + 1 < C) {
            const float up = (K + 2 < C) ? D[(K + 2 < C) ? K + 2 : K] : kInf;
            a_next = dtw_cost<P>(x0 - yv, min3f(D[(K + 1 < C) ? K + 1 : K], up, a_k));
        }
        const float b_k = dtw_cost<P>(x1 - yv, min3f(a_k, a_next, b_prev));
        D[K] = b_k;
        b_prev = b_k;
        a_k = a_next;
    }
}

// The abandon test after a row group (every 8 rows): the band's minimum, raised
// by the LB_Keogh terms of the rows not yet reached when `tail` (every path
// from the current row still crosses each later row i, at a cost of at least
// x_i's distance to the query envelope there, Sec. 7),
// against the threshold.  fp32: the two LB_Keogh sums (different orders) each
// carry at most n u relative error, and the path's remaining additions at
// most (2n - 1) u; c covers both.
__device__ __forceinline__ float raise_by_tail(float mn, int n, float lbk_total, float lbk_pre) {
    const float c = (float)(2 * n + 2) * 5.9604645e-8f;
    const float rest = fmaxf(0.0f, lbk_total - lbk_pre - c * lbk_total);
    return fmaxf(mn, (mn + rest) * (1.0f - c));
}

template <int C>
__device__ __forceinline__ bool reg4_abandons(const float (&D)[C], int n, bool tail, float lbk_total, float lbk_pre,
                                              float thr) {
    float mn = D[0];
#pragma unroll
    for (int k = 1; k < C; ++k) mn = fminf(mn, D[k]);
    if (tail) mn = raise_by_tail(mn, n, lbk_total, lbk_pre);
    return mn > thr;
}

// ---------------------------------------------------------------------------
// Register path: one thread per pair, the whole band of C = round_up(2w+1, 16)
// slots in registers.  The band occupies slots e..C-1 (e = C - (2w+1) < 16);
// slots below e are never written and stay +INF.  Each row enters the
// unrolled cell sequence at slot e (a jump on the uniform e).  The query band
// window is read from the four shifted copies with aligned 128-bit loads;
// when the 32 lanes of a warp share a query these are broadcasts.
// Pairs are taken 32 at a time from a global cursor (persistent grid).
// ---------------------------------------------------------------------------
template <int C, int P, int E>
__global__ void __launch_bounds__(kDtwThreads)
k_dtw_reg(DtwJob j, int e, int wl) {
    const int lane = threadIdx.x & 31;
    const int n = j.n;
    const int ylen = j.qc.ylen, padl = j.qc.padl;
    if (j.npairs_dev) j.npairs = (int64_t)*j.npairs_dev;
    const int wb = min(j.w, n - 1);
    const bool tail = (P == 1 || P == 2) && j.tU != nullptr && j.abandon;
    unsigned long long n_skip = 0, n_comp = 0, n_aband = 0, n_rows = 0, n_lane_rows = 0, n_cells = 0;
    for (;;) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(j.cursor, 1ull);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        const int64_t p0 = (int64_t)chunk * 32;
        if (p0 >= j.npairs) break;
        const int64_t pi = p0 + lane;
        int q, c;
        bool valid;
        fetch_pair(j, pi, q, c, valid);
        float thr = kInf;
        int my_rows = 0;
        if (valid) {
            thr = j.bsf ? load_threshold(j.bsf + q) : j.fixed_thr;
            if (j.pair_lbi && j.pair_lbi[pi] > thr * (1.0f + j.slack)) {
                j.res[pi] = kInf;
                valid = false;
                ++n_skip;
            }
        }
        if (valid) {
        ++n_comp;
        const float *x = j.db + (int64_t)c * n;
        const float *yc = j.qc.data + (int64_t)q * 4 * ylen;
        // the cumulative LB_Keogh abandon bound (Sec. 3 early abandoning with
        // the Sec. 7 terms of the rows still ahead): the pair's result
        // slot holds its LB_Keogh^p (read at each test, to spare registers),
        // and the terms of the rows passed so far are summed here; the rest
        // bounds the rows not yet reached
        const int64_t toff = tail ? (int64_t)q * n : 0;
        float lbk_pre = 0.0f;
        float D[C];
#pragma unroll
        for (int k = 0; k < C; ++k) D[k] = sel_eq(k, wl, 0.0f, kInf);  // row -1: D(-1,-1) = 0
        bool abandoned = false;
        int rows = n;
        int i = 0;
        if constexpr (E >= 0) {
            // two rows per step (reg_rows2), the abandon test after the same rows
            for (; i + 1 < n; i += 2) {
                const float x0 = __ldg(x + i), x1 = __ldg(x + i + 1);
                if (tail) {
                    lbk_pre = acc_dist<P>(lbk_pre, x0, __ldg(j.tL + toff + i), __ldg(j.tU + toff + i));
                    lbk_pre = acc_dist<P>(lbk_pre, x1, __ldg(j.tL + toff + i + 1), __ldg(j.tU + toff + i + 1));
                }
                reg_rows2<C, P, E>(D, x0, x1, yc, i, wl, padl, ylen);
                if (j.abandon && ((i + 1) & 7) == 7 && i + 2 < n) {
                    if (j.bsf) thr = load_threshold(j.bsf + q);
                    const float lbk_total = tail ? j.res[pi] : 0.0f;
                    if (reg4_abandons<C>(D, n, tail, lbk_total, lbk_pre, thr)) {
                        abandoned = true;
                        rows = i + 2;
                        break;
                    }
                }
            }
        }
        for (; !abandoned && i < n; ++i) {
            const float xi = __ldg(x + i);
            if (tail) lbk_pre = acc_dist<P>(lbk_pre, xi, __ldg(j.tL + toff + i), __ldg(j.tU + toff + i));
            reg_row<C, P>(D, xi, yc, i, e, wl, padl, ylen);
            if (j.abandon && (i & 7) == 7 && i + 1 < n) {
                if (j.bsf) thr = load_threshold(j.bsf + q);
                const float lbk_total = tail ? j.res[pi] : 0.0f;
                if (reg4_abandons<C>(D, n, tail, lbk_total, lbk_pre, thr)) {
                    abandoned = true;
                    rows = i + 1;
                    break;
                }
            }
        }
        n_rows += rows;
        my_rows = rows;
        n_cells += (unsigned long long)band_cells(rows, n, wb);
        float d = kInf;
#pragma unroll
        for (int k = 0; k < C; ++k) d = sel_eq(k, wl, D[k], d);
        if (abandoned) {
            d = kInf;
            ++n_aband;
        }
        if (!j.bsf && d > j.fixed_thr) d = kInf;
        j.res[pi] = j.root_out ? root_p(d, P) : d;
        if (!abandoned && j.bsf) update_threshold(j.bsf, j.gmin, j.k, q, c % j.k, d);
        }  // valid
        // the warp steps until its longest pair ends
        n_lane_rows += 32ull * __reduce_max_sync(0xffffffffu, (unsigned)my_rows);
    }
    if (j.counters) {
        // one atomic per warp and counter
        n_skip = __reduce_add_sync(0xffffffffu, (unsigned)n_skip);
        n_comp = __reduce_add_sync(0xffffffffu, (unsigned)n_comp);
        n_aband = __reduce_add_sync(0xffffffffu, (unsigned)n_aband);
        unsigned long long rows_w = 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n_rows += __shfl_xor_sync(0xffffffffu, n_rows, o);
        rows_w = n_rows;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n_cells += __shfl_xor_sync(0xffffffffu, n_cells, o);
        if (lane == 0) {
            if (rows_w) atomicAdd(j.counters + CNT_DTW_ROWS, rows_w);
            if (n_lane_rows) atomicAdd(j.counters + CNT_DTW_LANE_ROWS, n_lane_rows);
            if (n_cells) atomicAdd(j.counters + CNT_DTW_CELLS, n_cells);
            if (n_skip) atomicAdd(j.counters + CNT_DTW_SKIP, n_skip);
            if (n_comp) atomicAdd(j.counters + CNT_DTW_COMPUTED, n_comp);
            if (n_aband) atomicAdd(j.counters + CNT_DTW_ABANDONED, n_aband);
        }
    }
}

// ---------------------------------------------------------------------------
// Register path, 4 rows per window load (C <= 64).  Rows 4g .. 4g+3 need the
// query at padded indices 4g .. 4g + C + 2; with padl = wl that span starts
// on a 16-byte boundary of copy 0, so (C + 4) / 4 aligned 128-bit loads serve
// all four rows and row u's slot K reads window element u + K (a fixed
// register).  One 128-bit load of x covers the four rows.
// ---------------------------------------------------------------------------
template <int K, int C, int P, int U>
__device__ __forceinline__ void dtw_cells_win(float (&D)[C], float xi, const float (&yw)[C + 4]) {
    if constexpr (K < C) {
        dtw_cell<K, C, P>(D, xi, yw[U + K]);
        dtw_cells_win<K + 1, C, P, U>(D, xi, yw);
    }
}

// Cells K..C-1, two adjacent slots' differences per packed fma.
template <int K, int C, int P, int U>
__device__ __forceinline__ void dtw_cells_win2(float (&D)[C], float xi, const float (&yw)[C + 4]) {
    if constexpr (K + 1 < C) {
        const float2 d = dtw_diff2(xi, yw[U + K], yw[U + K + 1]);
        dtw_cell_d<K, C, P>(D, d.x);
        dtw_cell_d<K + 1, C, P>(D, d.y);
        dtw_cells_win2<K + 2, C, P, U>(D, xi, yw);
    } else if constexpr (K < C) {
        dtw_cell<K, C, P>(D, xi, yw[U + K]);
    }
}

// Cells K..C-1 of one row without a jump: used when the bottom padding E is
// a compile-time constant (the common bands), so that the rows of a group
// are one straight-line block the scheduler can interleave.
template <int C, int P, int U, int E>
__device__ __forceinline__ void dtw_row_win_fixed(float (&D)[C], float xi, const float (&yw)[C + 4]) {
    dtw_cells_win2<E, C, P, U>(D, xi, yw);
}

template <int C, int P, int U>
__device__ __forceinline__ void dtw_row_win(float (&D)[C], float xi, const float (&yw)[C + 4], int e) {
    switch (e) {
        case 0: dtw_cell<0, C, P>(D, xi, yw[U + 0]); [[fallthrough]];
        case 1: dtw_cell<1, C, P>(D, xi, yw[U + 1]); [[fallthrough]];
        case 2: dtw_cell<2, C, P>(D, xi, yw[U + 2]); [[fallthrough]];
        case 3: dtw_cell<3, C, P>(D, xi, yw[U + 3]); [[fallthrough]];
        case 4: dtw_cell<4, C, P>(D, xi, yw[U + 4]); [[fallthrough]];
        case 5: dtw_cell<5, C, P>(D, xi, yw[U + 5]); [[fallthrough]];
        case 6: dtw_cell<6, C, P>(D, xi, yw[U + 6]); [[fallthrough]];
        case 7: dtw_cell<7, C, P>(D, xi, yw[U + 7]); [[fallthrough]];
        case 8: dtw_cell<8, C, P>(D, xi, yw[U + 8]); [[fallthrough]];
        case 9: dtw_cell<9, C, P>(D, xi, yw[U + 9]); [[fallthrough]];
        case 10: dtw_cell<10, C, P>(D, xi, yw[U + 10]); [[fallthrough]];
        case 11: dtw_cell<11, C, P>(D, xi, yw[U + 11]); [[fallthrough]];
        case 12: dtw_cell<12, C, P>(D, xi, yw[U + 12]); [[fallthrough]];
        case 13: dtw_cell<13, C, P>(D, xi, yw[U + 13]); [[fallthrough]];
        case 14: dtw_cell<14, C, P>(D, xi, yw[U + 14]); [[fallthrough]];
        default: dtw_cell<15, C, P>(D, xi, yw[U + 15]);
    }
    dtw_cells_win<16, C, P, U>(D, xi, yw);
}

// Rows i .. i + 3 (those below n) of a thread-per-pair band, four rows per
// window load: the query window of the group read from copy 0 (y0 + i) with
// aligned 128-bit loads, x_i .. x_{i+3} with one (xvec) or four loads.  With
// `tail`, the LB_Keogh terms of these rows are added to lbk_pre when rows
// remain after them (the cumulative abandon bound of reg4_abandons).
template <int C, int P, int E>
__device__ __forceinline__ void reg4_rows(float (&D)[C], const float *__restrict__ x, const float *__restrict__ y0,
                                          int i, int n, int e, bool xvec, bool tail, const float *tu,
                                          const float *tl, float &lbk_pre) {
    float yw[C + 4];
    const float4 *yb = reinterpret_cast<const float4 *>(y0 + i);
#pragma unroll
    for (int v = 0; v < (C + 4) / 4; ++v) {
        const float4 t = __ldg(yb + v);
        yw[4 * v] = t.x;
        yw[4 * v + 1] = t.y;
        yw[4 * v + 2] = t.z;
        yw[4 * v + 3] = t.w;
    }
    float4 x4;
    if (xvec && i + 4 <= n) {
        x4 = __ldg(reinterpret_cast<const float4 *>(x + i));
    } else {
        x4.x = __ldg(x + i);
        x4.y = i + 1 < n ? __ldg(x + i + 1) : 0.0f;
        x4.z = i + 2 < n ? __ldg(x + i + 2) : 0.0f;
        x4.w = i + 3 < n ? __ldg(x + i + 3) : 0.0f;
    }
    if constexpr (E >= 0) {
        if (i + 4 <= n) {
            dtw_row_win_fixed<C, P, 0, E>(D, x4.x, yw);
            dtw_row_win_fixed<C, P, 1, E>(D, x4.y, yw);
            dtw_row_win_fixed<C, P, 2, E>(D, x4.z, yw);
            dtw_row_win_fixed<C, P, 3, E>(D, x4.w, yw);
        } else {
            dtw_row_win_fixed<C, P, 0, E>(D, x4.x, yw);
            if (i + 1 < n) dtw_row_win_fixed<C, P, 1, E>(D, x4.y, yw);
            if (i + 2 < n) dtw_row_win_fixed<C, P, 2, E>(D, x4.z, yw);
        }
    } else {
        dtw_row_win<C, P, 0>(D, x4.x, yw, e);
        if (i + 1 < n) dtw_row_win<C, P, 1>(D, x4.y, yw, e);
        if (i + 2 < n) dtw_row_win<C, P, 2>(D, x4.z, yw, e);
        if (i + 3 < n) dtw_row_win<C, P, 3>(D, x4.w, yw, e);
    }
    if (tail && i + 4 < n) {
        float4 u4, l4;
        if (xvec) {
            u4 = __ldg(reinterpret_cast<const float4 *>(tu + i));
            l4 = __ldg(reinterpret_cast<const float4 *>(tl + i));
        } else {
            u4 = make_float4(__ldg(tu + i), __ldg(tu + i + 1), __ldg(tu + i + 2), __ldg(tu + i + 3));
            l4 = make_float4(__ldg(tl + i), __ldg(tl + i + 1), __ldg(tl + i + 2), __ldg(tl + i + 3));
        }
        lbk_pre = acc_dist<P>(lbk_pre, x4.x, l4.x, u4.x);
        lbk_pre = acc_dist<P>(lbk_pre, x4.y, l4.y, u4.y);
        lbk_pre = acc_dist<P>(lbk_pre, x4.z, l4.z, u4.z);
        lbk_pre = acc_dist<P>(lbk_pre, x4.w, l4.w, u4.w);
    }
}

template <int C, int P, int E>
__global__ void __launch_bounds__(kDtwThreads)
k_dtw_reg4(DtwJob j, int e, int wl, bool xvec) {
    const int lane = threadIdx.x & 31;
    const int n = j.n;
    const int ylen = j.qc.ylen;
    if (j.npairs_dev) j.npairs = (int64_t)*j.npairs_dev;
    const int wb = min(j.w, n - 1);
    unsigned long long n_skip = 0, n_comp = 0, n_aband = 0, n_rows = 0, n_lane_rows = 0, n_cells = 0;
    for (;;) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(j.cursor, 1ull);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        const int64_t p0 = (int64_t)chunk * 32;
        if (p0 >= j.npairs) break;
        const int64_t pi = p0 + lane;
        int q, c;
        bool valid;
        fetch_pair(j, pi, q, c, valid);
        float thr = kInf;
        if (valid) {
            thr = j.bsf ? load_threshold(j.bsf + q) : j.fixed_thr;
            if (j.pair_lbi && j.pair_lbi[pi] > thr * (1.0f + j.slack)) {
                j.res[pi] = kInf;
                valid = false;
                ++n_skip;
            }
        }
        int my_rows = 0;
        if (valid) {
            ++n_comp;
            const float *x = j.db + (int64_t)c * n;
            const float *y0 = j.qc.data + (int64_t)q * 4 * ylen;  // copy 0; row i starts at index i
            float D[C];
#pragma unroll
            for (int k = 0; k < C; ++k) D[k] = sel_eq(k, wl, 0.0f, kInf);  // row -1: D(-1,-1) = 0
            bool abandoned = false;
            int rows = n;
            // Cumulative bound: after rows 0..i every warping path still
            // visits each later row k, at a cost of at least
            // d(x_k, [L_k, U_k])^p, so DTW^p >= (minimum of row i) + the
            // LB_Keogh^p terms of rows > i = LB_Keogh^p - those of rows <= i.
            const bool tail = (P == 1 || P == 2) && j.tU != nullptr && j.abandon;
            const float lbk_total = tail ? j.res[pi] : 0.0f;
            const float *tu = tail ? j.tU + (int64_t)q * n : nullptr;
            const float *tl = tail ? j.tL + (int64_t)q * n : nullptr;
            float lbk_pre = 0.0f;
            for (int i = 0; i < n; i += 4) {
                reg4_rows<C, P, E>(D, x, y0, i, n, e, xvec, tail, tu, tl, lbk_pre);
                if (j.abandon && (i & 4) && i + 4 < n) {
                    if (j.bsf) thr = load_threshold(j.bsf + q);
                    if (reg4_abandons<C>(D, n, tail, lbk_total, lbk_pre, thr)) {
                        abandoned = true;
                        rows = i + 4;
                        break;
                    }
                }
            }
            n_rows += rows;
            n_cells += (unsigned long long)band_cells(rows, n, wb);
            my_rows = rows;
            float d = kInf;
#pragma unroll
            for (int k = 0; k < C; ++k) d = sel_eq(k, wl, D[k], d);
            if (abandoned) {
                d = kInf;
                ++n_aband;
            }
            if (!j.bsf && d > j.fixed_thr) d = kInf;
            j.res[pi] = j.root_out ? root_p(d, P) : d;
            if (!abandoned && j.bsf) update_threshold(j.bsf, j.gmin, j.k, q, c % j.k, d);
        }  // valid
        // the warp steps until the chunk's longest pair ends
        n_lane_rows += 32ull * __reduce_max_sync(0xffffffffu, (unsigned)my_rows);
    }
    if (j.counters) {
        n_skip = __reduce_add_sync(0xffffffffu, (unsigned)n_skip);
        n_comp = __reduce_add_sync(0xffffffffu, (unsigned)n_comp);
        n_aband = __reduce_add_sync(0xffffffffu, (unsigned)n_aband);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n_rows += __shfl_xor_sync(0xffffffffu, n_rows, o);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n_cells += __shfl_xor_sync(0xffffffffu, n_cells, o);
        if (lane == 0) {
            if (n_rows) atomicAdd(j.counters + CNT_DTW_ROWS, n_rows);
            if (n_cells) atomicAdd(j.counters + CNT_DTW_CELLS, n_cells);
            if (n_skip) atomicAdd(j.counters + CNT_DTW_SKIP, n_skip);
            if (n_comp) atomicAdd(j.counters + CNT_DTW_COMPUTED, n_comp);
            if (n_aband) atomicAdd(j.counters + CNT_DTW_ABANDONED, n_aband);
            if (n_lane_rows) atomicAdd(j.counters + CNT_DTW_LANE_ROWS, n_lane_rows);
        }
    }
}

// ---------------------------------------------------------------------------
// Register path in row phases (C <= 64): the rows, cells, abandon test and
// results of k_dtw_reg4, but one launch evaluates only rows
// [row_begin, row_end) of its pairs.  A pair still alive at row_end (< n) is
// deferred: its band (the slots from e up; those below e are +INF padding)
// and LB_Keogh prefix are written to the out
// list, 32 consecutive pairs of a warp to consecutive entries, and the next
// launch resumes it from there.  A warp thus steps only until the longest of
// its pairs ends within the phase, and the next phase's warps are full again
// with pairs at the same row, so lanes idle for less than a phase; the
// pairs of a warp still share a row and mostly a query, so the query-window
// loads stay warp-wide broadcasts.  Listed pairs below *lead (every query's
// lowest-bound pairs, taken first) run to the last row in the first phase,
// so that thresholds fall before the bulk is resumed.  If the out list is
// full, the pair runs on in place.
// ---------------------------------------------------------------------------
template <int C, int P, int E>
__global__ void __launch_bounds__(kDtwThreads, (E >= 0 ? 3 : 2))
k_dtw_reg4p(DtwJob j, int e, int wl, bool xvec) {
    const int lane = threadIdx.x & 31;
    const int n = j.n;
    const int ylen = j.qc.ylen;
    const int wb = min(j.w, n - 1);
    const bool resume = j.ph.in_state != nullptr;
    const int64_t cap = j.ph.cap;
    int64_t npairs = j.npairs;
    if (resume) {
        const unsigned long long c_in = *j.ph.in_count;
        npairs = (int64_t)(c_in < (unsigned long long)cap ? c_in : (unsigned long long)cap);
    } else if (j.npairs_dev) {
        npairs = (int64_t)*j.npairs_dev;
    }
    const int64_t lead = (!resume && j.ph.lead) ? (int64_t)*j.ph.lead : 0;
    const int r0 = j.ph.row_begin;
    const int elo = E >= 0 ? E : e;  // lowest band slot
    const bool tail = (P == 1 || P == 2) && j.tU != nullptr && j.abandon;
    const unsigned long long cells0 = (unsigned long long)band_cells(r0, n, wb);
    unsigned long long n_skip = 0, n_comp = 0, n_aband = 0, n_rows = 0, n_lane_rows = 0, n_cells = 0;
    for (;;) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(j.cursor, 1ull);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        const int64_t p0 = (int64_t)chunk * 32;
        if (p0 >= npairs) break;
        const int64_t t = p0 + lane;
        bool alive = t < npairs;
        int64_t pi = 0;
        int q = 0, c = 0;
        if (alive) {
            pi = resume ? j.ph.in_pi[t] : t;
            const Pair pr = j.pairs[pi];
            q = pr.q;
            c = pr.c;
            if (c < 0) alive = false;
        }
        float thr = kInf;
        if (alive) {
            thr = j.bsf ? load_threshold(j.bsf + q) : j.fixed_thr;
            // a pair whose LB_Improved exceeds the threshold is skipped; a
            // resumed one, checked again against the threshold as it has
            // fallen since, is abandoned
            if (j.pair_lbi && j.pair_lbi[pi] > thr * (1.0f + j.slack)) {
                j.res[pi] = kInf;
                alive = false;
                if (resume)
                    ++n_aband;
                else
                    ++n_skip;
            }
        }
        if (alive && !resume) ++n_comp;
        // rows this lane runs to in this launch
        int stop = (pi < lead || j.ph.row_end >= n) ? n : j.ph.row_end;
        const float *x = j.db + (int64_t)c * n;
        const float *y0 = j.qc.data + (int64_t)q * 4 * ylen;  // copy 0; row i starts at index i
        const float *tu = tail ? j.tU + (int64_t)q * n : nullptr;
        const float *tl = tail ? j.tL + (int64_t)q * n : nullptr;
        const float lbk_total = (tail && alive) ? j.res[pi] : 0.0f;
        float D[C];
        float lbk_pre = 0.0f;
        if (resume) {
#pragma unroll
            for (int k = 0; k < C; ++k)  // the padding slots below e stay +INF and are not stored
                D[k] = (alive && k >= elo) ? j.ph.in_state[(int64_t)k * cap + t] : kInf;
            lbk_pre = alive ? j.ph.in_state[(int64_t)C * cap + t] : 0.0f;
        } else {
#pragma unroll
            for (int k = 0; k < C; ++k) D[k] = sel_eq(k, wl, 0.0f, kInf);  // row -1: D(-1,-1) = 0
        }
        bool abandoned = false, deferred = false;
        int i = r0;
        for (;;) {
            while (__any_sync(0xffffffffu, alive && i < stop)) {
                if (alive && i < stop) {
                    reg4_rows<C, P, E>(D, x, y0, i, n, e, xvec, tail, tu, tl, lbk_pre);
                    if (j.abandon && (i & 4) && i + 4 < n) {
                        if (j.bsf) thr = load_threshold(j.bsf + q);
                        if (reg4_abandons<C>(D, n, tail, lbk_total, lbk_pre, thr)) {
                            abandoned = true;
                            alive = false;
                        }
                    }
                    i += 4;
                }
            }
            // pairs alive at the end of the phase move to the out list
            const bool want = alive && stop < n;
            const unsigned m = __ballot_sync(0xffffffffu, want);
            if (m == 0) break;
            unsigned long long base = 0;
            const int leader = __ffs(m) - 1;
            if (lane == leader) base = atomicAdd(j.ph.out_count, (unsigned long long)__popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (want) {
                const int64_t slot = (int64_t)base + __popc(m & ((1u << lane) - 1));
                if (slot < cap) {
#pragma unroll
                    for (int k = 0; k < C; ++k)
                        if (k >= elo) j.ph.out_state[(int64_t)k * cap + slot] = D[k];
                    j.ph.out_state[(int64_t)C * cap + slot] = lbk_pre;
                    j.ph.out_pi[slot] = pi;
                    deferred = true;
                    alive = false;
                } else {
                    stop = n;  // no room: this pair runs on here
                }
            }
            if (!__any_sync(0xffffffffu, alive && i < stop)) break;
        }
        const int rows = min(i, n);  // rows evaluated so far (abandoned pairs: through their last group)
        if (i > r0) {
            n_rows += (unsigned long long)(rows - r0);
            n_cells += (unsigned long long)band_cells(rows, n, wb) - cells0;
        }
        n_lane_rows += 32ull * __reduce_max_sync(0xffffffffu, (unsigned)(i > r0 ? min(i, n) - r0 : 0));
        if (abandoned) {
            ++n_aband;
            j.res[pi] = kInf;
        } else if (alive) {
            // completed: the last row was evaluated
            float d = kInf;
#pragma unroll
            for (int k = 0; k < C; ++k) d = sel_eq(k, wl, D[k], d);
            if (!j.bsf && d > j.fixed_thr) d = kInf;
            j.res[pi] = j.root_out ? root_p(d, P) : d;
            if (j.bsf) update_threshold(j.bsf, j.gmin, j.k, q, c % j.k, d);
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
            if (n_rows) atomicAdd(j.counters + CNT_DTW_ROWS, n_rows);
            if (n_cells) atomicAdd(j.counters + CNT_DTW_CELLS, n_cells);
            if (n_skip) atomicAdd(j.counters + CNT_DTW_SKIP, n_skip);
            if (n_comp) atomicAdd(j.counters + CNT_DTW_COMPUTED, n_comp);
            if (n_aband) atomicAdd(j.counters + CNT_DTW_ABANDONED, n_aband);
            if (n_lane_rows) atomicAdd(j.counters + CNT_DTW_LANE_ROWS, n_lane_rows);
        }
    }
}

// The register path of bands wider than 64 slots (k_dtw_reg's rows, one per
// step, abandon test every 8 rows) in row phases, with the continuation
// lists, leading region and deferral of k_dtw_reg4p.
template <int C, int P>
__global__ void __launch_bounds__(kDtwThreads, (C <= 112 ? 3 : 2))
k_dtw_regp(DtwJob j, int e, int wl) {
    const int lane = threadIdx.x & 31;
    const int n = j.n;
    const int ylen = j.qc.ylen, padl = j.qc.padl;
    const int wb = min(j.w, n - 1);
    const bool resume = j.ph.in_state != nullptr;
    const int64_t cap = j.ph.cap;
    int64_t npairs = j.npairs;
    if (resume) {
        const unsigned long long c_in = *j.ph.in_count;
        npairs = (int64_t)(c_in < (unsigned long long)cap ? c_in : (unsigned long long)cap);
    } else if (j.npairs_dev) {
        npairs = (int64_t)*j.npairs_dev;
    }
    const int64_t lead = (!resume && j.ph.lead) ? (int64_t)*j.ph.lead : 0;
    const int r0 = j.ph.row_begin;
    const int elo = e;  // lowest band slot
    const bool tail = (P == 1 || P == 2) && j.tU != nullptr && j.abandon;
    const unsigned long long cells0 = (unsigned long long)band_cells(r0, n, wb);
    unsigned long long n_skip = 0, n_comp = 0, n_aband = 0, n_rows = 0, n_lane_rows = 0, n_cells = 0;
    for (;;) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(j.cursor, 1ull);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        const int64_t p0 = (int64_t)chunk * 32;
        if (p0 >= npairs) break;
        const int64_t t = p0 + lane;
        bool alive = t < npairs;
        int64_t pi = 0;
        int q = 0, c = 0;
        if (alive) {
            pi = resume ? j.ph.in_pi[t] : t;
            const Pair pr = j.pairs[pi];
            q = pr.q;
            c = pr.c;
            if (c < 0) alive = false;
        }
        float thr = kInf;
        if (alive) {
            thr = j.bsf ? load_threshold(j.bsf + q) : j.fixed_thr;
            // a pair whose LB_Improved exceeds the threshold is skipped; a
            // resumed one, checked again against the threshold as it has
            // fallen since, is abandoned
            if (j.pair_lbi && j.pair_lbi[pi] > thr * (1.0f + j.slack)) {
                j.res[pi] = kInf;
                alive = false;
                if (resume)
                    ++n_aband;
                else
                    ++n_skip;
            }
        }
        if (alive && !resume) ++n_comp;
        int stop = (pi < lead || j.ph.row_end >= n) ? n : j.ph.row_end;
        const float *x = j.db + (int64_t)c * n;
        const float *yc = j.qc.data + (int64_t)q * 4 * ylen;
        const int64_t toff = tail ? (int64_t)q * n : 0;
        float D[C];
        float lbk_pre = 0.0f;
        if (resume) {
#pragma unroll
            for (int k = 0; k < C; ++k)  // the padding slots below e stay +INF and are not stored
                D[k] = (alive && k >= elo) ? j.ph.in_state[(int64_t)k * cap + t] : kInf;
            lbk_pre = alive ? j.ph.in_state[(int64_t)C * cap + t] : 0.0f;
        } else {
#pragma unroll
            for (int k = 0; k < C; ++k) D[k] = sel_eq(k, wl, 0.0f, kInf);  // row -1: D(-1,-1) = 0
        }
        bool abandoned = false;
        int i = r0;
        for (;;) {
            while (__any_sync(0xffffffffu, alive && i < stop)) {
                if (alive && i < stop) {
                    const float xi = __ldg(x + i);
                    if (tail) lbk_pre = acc_dist<P>(lbk_pre, xi, __ldg(j.tL + toff + i), __ldg(j.tU + toff + i));
                    reg_row<C, P>(D, xi, yc, i, e, wl, padl, ylen);
                    if (j.abandon && (i & 7) == 7 && i + 1 < n) {
                        if (j.bsf) thr = load_threshold(j.bsf + q);
                        const float lbk_total = tail ? j.res[pi] : 0.0f;
                        if (reg4_abandons<C>(D, n, tail, lbk_total, lbk_pre, thr)) {
                            abandoned = true;
                            alive = false;
                        }
                    }
                    ++i;
                }
            }
            // pairs alive at the end of the phase move to the out list
            const bool want = alive && stop < n;
            const unsigned m = __ballot_sync(0xffffffffu, want);
            if (m == 0) break;
            unsigned long long base = 0;
            const int leader = __ffs(m) - 1;
            if (lane == leader) base = atomicAdd(j.ph.out_count, (unsigned long long)__popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (want) {
                const int64_t slot = (int64_t)base + __popc(m & ((1u << lane) - 1));
                if (slot < cap) {
#pragma unroll
                    for (int k = 0; k < C; ++k)
                        if (k >= elo) j.ph.out_state[(int64_t)k * cap + slot] = D[k];
                    j.ph.out_state[(int64_t)C * cap + slot] = lbk_pre;
                    j.ph.out_pi[slot] = pi;
                    alive = false;
                } else {
                    stop = n;  // no room: this pair runs on here
                }
            }
            if (!__any_sync(0xffffffffu, alive && i < stop)) break;
        }
        const int rows = min(i, n);
        if (i > r0) {
            n_rows += (unsigned long long)(rows - r0);
            n_cells += (unsigned long long)band_cells(rows, n, wb) - cells0;
        }
        n_lane_rows += 32ull * __reduce_max_sync(0xffffffffu, (unsigned)(i > r0 ? rows - r0 : 0));
        if (abandoned) {
            ++n_aband;
            j.res[pi] = kInf;
        } else if (alive) {
            float d = kInf;
#pragma unroll
            for (int k = 0; k < C; ++k) d = sel_eq(k, wl, D[k], d);
            if (!j.bsf && d > j.fixed_thr) d = kInf;
            j.res[pi] = j.root_out ? root_p(d, P) : d;
            if (j.bsf) update_threshold(j.bsf, j.gmin, j.k, q, c % j.k, d);
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
            if (n_rows) atomicAdd(j.counters + CNT_DTW_ROWS, n_rows);
            if (n_cells) atomicAdd(j.counters + CNT_DTW_CELLS, n_cells);
            if (n_skip) atomicAdd(j.counters + CNT_DTW_SKIP, n_skip);
            if (n_comp) atomicAdd(j.counters + CNT_DTW_COMPUTED, n_comp);
            if (n_aband) atomicAdd(j.counters + CNT_DTW_ABANDONED, n_aband);
            if (n_lane_rows) atomicAdd(j.counters + CNT_DTW_LANE_ROWS, n_lane_rows);
        }
    }
}

// ---------------------------------------------------------------------------
// Wide path (2w+1 > 208): one warp per pair, lane l owns the CL slots
// l*CL .. l*CL+CL-1 of the band (slot k holds column i - w + k; slots above
// 2w are outside the band).  A slot depends on the slot below it in the same
// row and on the slot above it in the previous row, so lane l computes row i
// at step t = 2i + l: the left neighbour finished row i and the right
// neighbour finished row i-1 one step earlier, and their boundary values
// arrive by shuffles.  The lane that holds slot 2w+1 resets it to +INF after
// each row so that the band's top edge reads +INF.  Each lane keeps its
// window of the query in registers and slides it by one column per row.
// The row minimum is carried along the lanes with the boundary values; the
// lane holding slot 2w sees the full minimum of its row.
// ---------------------------------------------------------------------------
template <int CL, int P>
__global__ void __launch_bounds__(kDtwThreads)
k_dtw_wide(DtwJob j) {
    const int lane = threadIdx.x & 31;
    const int n = j.n;
    const int w = min(j.w, n - 1);
    const int padl = j.qc.padl;
    const int top = 2 * w;             // highest band slot
    const int lane_top = top / CL;     // lane holding slot 2w
    const int lane_dead = (top + 1) / CL, c_dead = (top + 1) % CL;  // slot 2w+1
    const int lane_diag = w / CL, c_diag = w % CL;                  // slot of column i
    if (j.npairs_dev) j.npairs = (int64_t)*j.npairs_dev;
    unsigned long long n_skip = 0, n_comp = 0, n_aband = 0, n_rows = 0, n_cells = 0;
    for (;;) {
        unsigned long long pw = 0;
        if (lane == 0) pw = atomicAdd(j.cursor, 1ull);
        pw = __shfl_sync(0xffffffffu, pw, 0);
        const int64_t pi = (int64_t)pw;
        if (pi >= j.npairs) break;
        int q, c;
        bool valid;
        fetch_pair(j, pi, q, c, valid);
        float thr = kInf;
        if (valid) {
            thr = j.bsf ? load_threshold(j.bsf + q) : j.fixed_thr;
            if (j.pair_lbi && j.pair_lbi[pi] > thr * (1.0f + j.slack)) {
                if (lane == 0) {
                    j.res[pi] = kInf;
                    ++n_skip;
                }
                valid = false;
            }
        }
        if (!valid) continue;  // uniform across the warp
        if (lane == 0) ++n_comp;
        const float *x = j.db + (int64_t)c * n;
        const float *yp = j.qc.data + (int64_t)q * 4 * j.qc.ylen + padl;  // copy 0, column 0
        float D[CL], yw[CL];
        const int k0 = lane * CL;
#pragma unroll
        for (int t = 0; t < CL; ++t) {
            D[t] = sel_eq(k0 + t, w, 0.0f, kInf);  // row -1: D(-1,-1) = 0
            yw[t] = __ldg(yp + (0 - w + k0 + t));  // window of row 0
        }
        float ex_first = D[0], ex_last = D[CL - 1], ex_min = kInf;
        bool abandoned = false;
        const int steps = 2 * (n - 1) + 32;
        for (int t = 0; t < steps; ++t) {
            float left = __shfl_up_sync(0xffffffffu, ex_last, 1);
            float up = __shfl_down_sync(0xffffffffu, ex_first, 1);
            float lmin = __shfl_up_sync(0xffffffffu, ex_min, 1);
            if (lane == 0) {
                left = kInf;
                lmin = kInf;
            }
            if (lane == 31) up = kInf;
            const int dd = t - lane;
            if (dd >= 0 && !(dd & 1) && (dd >> 1) < n && lane <= lane_dead) {
                const int i = dd >> 1;
                if (i > 0) {
#pragma unroll
                    for (int u = 0; u + 1 < CL; ++u) yw[u] = yw[u + 1];
                    yw[CL - 1] = __ldg(yp + (i - w + k0 + CL - 1));
                }
                const float xi = __ldg(x + i);
                float mn = kInf;
#pragma unroll
                for (int u = 0; u < CL; ++u) {
                    const float above = (u + 1 < CL) ? D[(u + 1 < CL) ? u + 1 : u] : up;
                    const float below = (u > 0) ? D[(u > 0) ? u - 1 : 0] : left;
                    const float m = min3f(D[u], above, below);
                    const float df = xi - yw[u];
                    D[u] = dtw_cost<P>(df, m);
                    mn = fminf(mn, D[u]);
                }
                if (lane == lane_dead) {
                    // slot 2w+1 lies outside the band
#pragma unroll
                    for (int u = 0; u < CL; ++u) D[u] = sel_eq(u, c_dead, kInf, D[u]);
                }
                ex_first = D[0];
                ex_last = D[CL - 1];
                ex_min = (lane <= lane_top) ? fminf(mn, lmin) : lmin;
            }
            if (j.abandon && (t & 7) == 7 && t >= lane_top) {
                // lane_top has completed at least row 0, so its running
                // minimum covers a whole row
                const float rowmin = __shfl_sync(0xffffffffu, ex_min, lane_top);
                if (j.bsf) thr = load_threshold(j.bsf + q);
                thr = __shfl_sync(0xffffffffu, thr, 0);
                if (rowmin > thr) {  // uniform: every lane sees lane_top's value
                    abandoned = true;
                    const int rows = max(0, min(n, (t - lane_top) / 2 + 1));
                    n_rows += (unsigned long long)rows;
                    n_cells += (unsigned long long)band_cells(rows, n, w);
                    break;
                }
            }
        }
        if (!abandoned) {
            n_rows += (unsigned long long)n;
            n_cells += (unsigned long long)band_cells(n, n, w);
        }
        float dv = kInf;
#pragma unroll
        for (int u = 0; u < CL; ++u) dv = sel_eq(u, c_diag, D[u], dv);
        dv = __shfl_sync(0xffffffffu, dv, lane_diag);
        if (abandoned) dv = kInf;
        if (lane == 0) {
            if (abandoned) ++n_aband;
            if (!j.bsf && dv > j.fixed_thr) dv = kInf;
            j.res[pi] = j.root_out ? root_p(dv, P) : dv;
            if (!abandoned && j.bsf) update_threshold(j.bsf, j.gmin, j.k, q, c % j.k, dv);
        }
    }
    if (j.counters && lane == 0) {
        if (n_rows) atomicAdd(j.counters + CNT_DTW_ROWS, n_rows);
        if (n_cells) atomicAdd(j.counters + CNT_DTW_CELLS, n_cells);
        if (n_skip) atomicAdd(j.counters + CNT_DTW_SKIP, n_skip);
        if (n_comp) atomicAdd(j.counters + CNT_DTW_COMPUTED, n_comp);
        if (n_aband) atomicAdd(j.counters + CNT_DTW_ABANDONED, n_aband);
    }
}

}  // namespace dtwk

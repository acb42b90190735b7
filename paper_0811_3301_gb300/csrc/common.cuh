// Shared device helpers and internal launcher declarations of the DTW cascade
// library (sm_103a).  Internal: the public ABI is include/dtwknn.h.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/dtwknn.h"

namespace dtwk {

constexpr float kInf = __builtin_huge_valf();

// Three-input fp32 min/max (PTX ISA 8.8, sm_100+).  NaN-free inputs only.
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// (k == m) ? a : b, written in PTX so that loops of such selects over a
// register array are not folded into a dynamically indexed (local-memory)
// access by the optimiser.
__device__ __forceinline__ float sel_eq(int k, int m, float a, float b) {
    float r;
    asm("{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %1, %2;\n\tselp.f32 %0, %3, %4, p;\n\t}"
        : "=f"(r)
        : "r"(k), "r"(m), "f"(a), "f"(b));
    return r;
}

// Distance from v to the interval [lo, hi] (lo <= hi), raised to the power P:
// the per-index term of LB_Keogh (Sec. 7, Eq. 1): |v - H_i|^P.
template <int P>
__device__ __forceinline__ float dist_pow(float v, float lo, float hi) {
    float d = max3f(v - hi, lo - v, 0.0f);
    return P == 1 ? d : d * d;
}
template <int P>
__device__ __forceinline__ float acc_dist(float acc, float v, float lo, float hi) {
    float d = max3f(v - hi, lo - v, 0.0f);
    return P == 1 ? acc + d : fmaf(d, d, acc);
}

// Root of a power-space value (the paper's DTW_p and LB_p carry the root);
// p = 0 stands for p = infinity, whose values carry no power.
__device__ __forceinline__ float root_p(float v, int p) {
    return (p == 1 || p == 0) ? v : (p == 2 ? sqrtf(v) : sqrtf(sqrtf(v)));
}

// One band cell of DTW_p (Sec. 4): the cost of (x_i, y_j) combined with the
// best predecessor m.  P = 1, 2, 4: m + |d|^P (a sum along the path; the
// result is DTW_P^P); P = 0 (p = infinity): max(|d|, m) (the largest cost
// along the path).  Both never decrease m, which early abandoning relies on.
template <int P>
__device__ __forceinline__ float dtw_cost(float d, float m) {
    static_assert(P == 0 || P == 1 || P == 2 || P == 4, "p in {1, 2, 4, infinity}");
    if constexpr (P == 1) return fabsf(d) + m;
    if constexpr (P == 2) return fmaf(d, d, m);
    if constexpr (P == 4) {
        const float s = d * d;
        return fmaf(s, s, m);
    }
    return fmaxf(fabsf(d), m);
}

__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

// Four consecutive bound terms d(v, [lo, hi])^P added to acc.
template <int P>
__device__ __forceinline__ float acc_dist4(float acc, float4 v, float4 lo, float4 hi) {
    acc = acc_dist<P>(acc, v.x, lo.x, hi.x);
    acc = acc_dist<P>(acc, v.y, lo.y, hi.y);
    acc = acc_dist<P>(acc, v.z, lo.z, hi.z);
    return acc_dist<P>(acc, v.w, lo.w, hi.w);
}
__device__ __forceinline__ float4 min4(float4 a, float4 b) {
    return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), fminf(a.w, b.w));
}
__device__ __forceinline__ float4 max4(float4 a, float4 b) {
    return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z), fmaxf(a.w, b.w));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Indices between the partial-sum tests of the filter's early abandoning.
constexpr int kLbAbandonSpan = 256;

// Pairs per warp whose bound sums are reduced together (warp_sum16_transposed).
constexpr int kLbiBatch = 8;

// v[16] over the warp (a transposed butterfly: each exchange step halves the
// values a lane holds): lane l returns the warp sum of v[(l >> 1) & 15].
__device__ __forceinline__ float warp_sum16_transposed(float (&v)[16]) {
    const int lane = threadIdx.x & 31;
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float send = b4 ? v[i] : v[i + 8];
        const float keep = b4 ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = b3 ? v[i] : v[i + 4];
        const float keep = b3 ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b2 ? v[i] : v[i + 2];
        const float keep = b2 ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    float r = (b1 ? v[1] : v[0]) + __shfl_xor_sync(0xffffffffu, b1 ? v[0] : v[1], 2);
    return r + __shfl_xor_sync(0xffffffffu, r, 1);
}

// Non-negative floats order like their bit patterns; +INF is 0x7f800000.
__device__ __forceinline__ float load_threshold(const uint32_t *bits) {
    return __uint_as_float(*(volatile const uint32_t *)bits);
}

// Worst-case relative fp32 rounding of the quantities compared by the
// pruning tests (derivation in the design notes): an LB sum of up to 2n
// terms and a DTW path sum of up to 2n - 1 cells, each term rounded once.
__host__ __device__ inline float auto_slack(int n) {
    const double u = 5.9604644775390625e-8;  // 2^-24
    return (float)((4.0 * n + 16.0) * u * 1.0625);
}

// ---------------------------------------------------------------------------
// Per-query preprocessed data used by the DTW kernels: four copies of the
// query padded with +INF on both sides and shifted by 0..3 elements, so that
// any band window starts on a 16-byte boundary in one of the copies.
//   ycopy[(q * 4 + r) * ylen + t] = ypad(t + r - padl),
//   ypad(j) = y[j] for 0 <= j < n, +INF otherwise.
// ---------------------------------------------------------------------------
struct QueryCopies {
    float *data = nullptr;
    int padl = 0;   // multiple of 4
    int ylen = 0;   // multiple of 4
};


// ---------------------------------------------------------------------------
// Launchers (all asynchronous on `s`; they return cudaGetLastError()).
// ---------------------------------------------------------------------------
// U, L of count series (and, with UL/LU, the second-order envelopes
// UL = U(L), LU = L(U)); qc.data: optional shifted copies.
cudaError_t launch_envelope(const float *y, int64_t count, int n, int w, float *U, float *L,
                            QueryCopies qc, int copies_padl, cudaStream_t s, float *UL = nullptr,
                            float *LU = nullptr);

cudaError_t launch_lbk_single(const float *cand, int64_t N, const float *U, const float *L, int n,
                              int p, float *out, cudaStream_t s);
cudaError_t launch_lbk_tile(const float *db, int N, const float *U, const float *L, int Q, int n,
                            int p, float *lb, unsigned long long *tile_min, cudaStream_t s);
int lbk_tiles(int N);  // candidate tiles of the all-pairs kernel

// Piecewise-sum bound (Sec. 9): cover of d parts, floor(n/d) indices each,
// the last part takes the rest.
struct PartGeom {
    int d, s, smax;
};
inline PartGeom part_geom(int n, int d) {
    PartGeom g;
    g.d = d;
    g.s = n / d;
    g.smax = n - (d - 1) * g.s;
    return g;
}
// PX[c][j] = sum of db row c over part j; xmax_bits = max |x| (float bits).
cudaError_t launch_summarize(const float *db, int64_t N, int n, int d, float *PX, unsigned *xmax_bits,
                             cudaStream_t s);
// PU[q][j], PL[q][j]: part sums of U and L, widened (when widen != 0) by the
// worst-case fp32 rounding of the part sums so the fp32 bound never exceeds
// the exact one.
cudaError_t launch_query_summary(const float *U, const float *L, int64_t Q, int n, int d,
                                 const unsigned *xmax_bits, float *PU, float *PL, int widen, cudaStream_t s);
cudaError_t launch_lbp_single(const float *cand, int64_t N, const float *U, const float *L, int n, int d, int p,
                              float *out, float *scratch, cudaStream_t s);

// One (query, candidate) pair for the LB_Improved and DTW stages.
struct Pair {
    int32_t q;
    int32_t c;
};

// LB_Improved^(1/p) of cand [N][n] against q [n] with envelope U, L, from the
// candidates' envelopes XU, XL [N][n] and the query's U(L), L(U) [n] (same band).
cudaError_t launch_lbi_single(const float *cand, int64_t N, const float *q, const float *U, const float *L,
                              const float *XU, const float *XL, const float *UL, const float *LU, int n, int p,
                              float *out, cudaStream_t s);

struct CascadeBufs {
    // inputs
    const float *db;        // [N][n]
    const float *queries;   // [Q][n]
    const float *U, *L;     // [Q][n]
    const float *UL, *LU;   // [Q][n] U(L) and L(U), for LB_Improved's second sum
    const float *XU, *XL;   // [N][n] the candidates' own envelopes (same band)
    QueryCopies qc;
    int N, Q, n, w, p, k, mode;
    float slack;
    // LB_Keogh matrix, [Q][N], power space, and per (query, tile) minimum keys
    float *lb;
    unsigned long long *tile_min;  // [Q][ntiles]
    int ntiles;
    // seeds: [Q][S]
    int S;
    Pair *seed_pairs;
    float *seed_res;
    // thresholds: group minima [Q][k] and the bound [Q], float bits
    uint32_t *gmin;
    uint32_t *bsf;
    // survivors of the bound stages, as written by the filter (unordered) ...
    Pair *pairs_u;
    float *lbi_u;
    // ... and grouped by query, each pair's result slot holding its
    // LB_Keogh^p (from the matrix, where the filter leaves it for its
    // survivors) until the DTW stage writes the result.  With order_first = F > 0 each query's pairs
    // are ordered by ascending bound (to 1/256 of its threshold) and split:
    // its first min(F, qcount[q]) pairs at qstart[q] in a leading region that
    // holds every query's first pairs, the rest at qstart_b[q] after it.  With
    // F = 0 query q owns [qstart[q], qstart[q] + qcount[q]) in filter order.
    Pair *pairs;
    float *pair_lbi;
    float *pair_res;
    int32_t *qcount;      // [Q], zeroed before the filter
    int32_t *qstart;      // [Q]
    int32_t *qstart_b;    // [Q], used when order_first > 0
    int order_first;
    unsigned long long *pair_total;  // pairs after grouping
    unsigned long long *lead_total;  // pairs in the leading region (order_first > 0), else 0
    int lbi_inline;       // the filter computes LB_Improved (warp per pair)
    int summary;          // the matrix holds the piecewise-sum bound; LB_Keogh is computed in the filter
    float summary_scale;  // max_j |C_j| for p = 2 (matrix units), 1 for p = 1
    int64_t pair_cap;
    unsigned long long *pair_count;
    int seg_len, nseg;    // nseg: sub-segments per query (segments x filter warps)
    int seg_per_cta;      // consecutive segments one filter CTA handles
    int filter_warps;     // warps per filter CTA (one sub-segment each)
    int filter_path;      // 1 one warp per pair, 2 batches of eight pairs per warp (resolved by the plan)
    int lb_abandon;       // streamed long rows: stop a pair's sums once their partial values exceed thr
    unsigned *dev_err;    // a kernel's bounded wait that gave up records its dtw_status here (0: none)
    int32_t *seg_start;   // [Q][nseg]
    int32_t *seg_count;   // [Q][nseg]
    // work cursors and counters
    unsigned long long *cursor;       // DTW chunk cursor
    unsigned long long *counters;     // 8 counters, see dtw_stats
    // outputs (device)
    int64_t *out_idx;
    float *out_dist;
};

cudaError_t launch_seed_select(const CascadeBufs &b, cudaStream_t s);
cudaError_t launch_seed_kth(const CascadeBufs &b, cudaStream_t s);
cudaError_t launch_query_copies(const float *y, int64_t count, int n, QueryCopies qc, cudaStream_t s);
cudaError_t launch_lbi_filter(const CascadeBufs &b, cudaStream_t s);
// warps per filter CTA (one sub-segment each): `want` (1..8) if its shared
// memory fits a CTA, else fewer; want = 0 chooses from the occupancy
int lbi_filter_warps(int n, int w, int S, int seg_len, int p, int want = 0);
// The batched filter (filter_path 2) serves series of 128 or 256 elements
// with the piecewise-sum pre-filter and LB_Improved on.
bool lbi_batch_applies(int n, bool summary, bool lbi_inline);
cudaError_t launch_finalize(const CascadeBufs &b, cudaStream_t s);
// bsf[q] = min(bsf[q], thr_in[q]) (thr_in nullable; has_db false: no
// database, the threshold is +INF and bsf is not touched), then thr_out[q] =
// bsf[q] (nullable); Q thresholds, power space.
cudaError_t launch_threshold_io(uint32_t *bsf, int Q, bool has_db, const float *thr_in, float *thr_out,
                                cudaStream_t s);
// The k smallest (distance, index) of R per-shard lists [R][Q][k_in] per query.
cudaError_t launch_merge_topk(const int64_t *idx, const float *dist, int R, int Q, int k_in, int k,
                              int64_t *out_idx, float *out_dist, cudaStream_t s);
cudaError_t launch_group_by_query(const CascadeBufs &b, cudaStream_t s);


// DTW over an explicit pair list (pairs != nullptr) or the implicit pairs
// c -> (q = per_pair_y ? c : 0, c).  thr_bits: per-query thresholds (float
// bits, power space) read live for early abandoning, or nullptr with a fixed
// power-space threshold fixed_thr.  res receives DTW^p or +INF.
struct DtwJob {
    const float *db;
    int n, w, p, k;
    QueryCopies qc;
    const Pair *pairs;        // or nullptr
    int64_t npairs;           // pair count, or the upper bound when npairs_dev is set
    const unsigned long long *npairs_dev;  // nullable: pair count in device memory
    int per_pair_y;           // implicit pairs: query index = pair index
    const float *pair_lbi;    // nullable: skip a pair whose bound exceeds the live threshold
    float slack;
    uint32_t *bsf;            // nullable: live per-query threshold (updated on completion)
    uint32_t *gmin;           // nullable: per-query group minima [Q][k]
    float fixed_thr;          // used when bsf == nullptr
    int abandon;              // 0: never abandon
    float *res;               // [npairs]
    int root_out;             // store DTW_p (root taken) instead of DTW_p^p
    unsigned long long *cursor;    // chunk cursor (zeroed by the caller)
    unsigned long long *counters;  // nullable
    int lanes;                // 1: warp path (lane groups share a pair's band); 2: with 16-lane groups
    // Cumulative LB_Keogh in the abandon test (thread-per-pair kernel): res
    // holds each listed pair's LB_Keogh^p on entry, tU/tL [Q][n] the query
    // envelopes.  nullptr: the row minimum alone.
    const float *tU, *tL;
    // Row phases of the thread-per-pair register kernel (k_dtw_reg4p): the
    // launch evaluates rows [row_begin, row_end) of its pairs; a pair still
    // alive at row_end < n is deferred: its band state goes to the out list
    // and the next launch resumes it.  Pairs read from an in list (in_state
    // != nullptr) resume at row_begin; listed pairs whose index is below
    // *lead run to the last row in the first launch.
    struct Phase {
        int row_begin, row_end;
        const unsigned long long *lead;
        // lists, structure of arrays: state[k * cap + t] (band slots k < C,
        // then the LB_Keogh prefix at k = C), pi[t] the pair's list index
        const float *in_state;
        const int64_t *in_pi;
        const unsigned long long *in_count;
        float *out_state;
        int64_t *out_pi;
        unsigned long long *out_count;
        int64_t cap;
    } ph;
};


// counters layout
enum {
    CNT_KEOGH_PASS = 0,     // non-seed pairs with LB_Keogh^p <= thr
    CNT_LBI_PASS = 1,       // pairs written to the DTW list
    CNT_DTW_SKIP = 2,       // listed pairs skipped because the live threshold fell below their bound
    CNT_DTW_COMPUTED = 3,   // listed pairs whose DTW was started
    CNT_DTW_ABANDONED = 4,  // of which abandoned early
    CNT_DTW_ROWS = 5,       // DP rows evaluated
    CNT_SUMMARY_PASS = 6,   // non-seed pairs with piecewise-sum bound <= thr
    CNT_DTW_LANE_ROWS = 7,  // thread-per-pair DTW: 32 x the longest pair's rows, per chunk of 32
    CNT_DTW_CELLS = 8,      // in-band cells of the DP rows evaluated (band_cells per pair)
    CNT_NUM = 9
};
// A run's counter block: CNT_NUM run counters, CNT_NUM seed-stage counters,
// then one word where a kernel whose bounded wait gave up records its
// dtw_status (0: none).
constexpr int CNT_ERR = 2 * CNT_NUM;
constexpr int CNT_ALLOC = 2 * CNT_NUM + 1;

// In-band cells of rows 0..r-1 of the band DTW (|i - j| <= w, 0 <= j < n):
// row i holds min(n - 1, i + w) - max(0, i - w) + 1 cells.  In closed form,
// sum_{i<r} min(n, i + w + 1) - sum_{i<r} max(0, i - w); r = n gives
// n (2w + 1) - w (w + 1) for w <= n - 1.
__host__ __device__ inline long long tri_num(long long m) { return m > 0 ? m * (m + 1) / 2 : 0LL; }
__host__ __device__ inline long long band_cells(long long r, long long n, long long w) {
    if (r <= 0) return 0;
    return r * (r - 1) / 2 + r * (w + 1) - tri_num(r - n + w) - tri_num(r - 1 - w);
}

int device_sm_count();

// Host-side argument handling shared by entry points in several translation
// units (api.cu).  fail() records the calling thread's dtw_last_error message
// and returns st.
dtw_status fail(dtw_status st, const char *fmt, ...);
// The checks of dtw_band's arguments (n, w, p, the band width, N, y_stride,
// the threshold, the pointers); DTW_OK with *empty = true when N == 0.
dtw_status check_dtw_band_args(const float *x, const float *y, int64_t N, int32_t y_stride, int32_t n, int32_t w,
                               int32_t p, float threshold, const float *out, bool *empty);
// A threshold on DTW_p in the units the kernels compare (DTW_p^p; DTW_inf itself).
float threshold_power(float t, int32_t p);

cudaError_t launch_triangle_ratio(const float *dxy, const float *dyz, const float *dxz, int64_t N, float *out,
                                  cudaStream_t s);

}  // namespace dtwk

// Persistent form of the mixed-length batch: one launch over a device work
// queue of (group, query, candidate chunk) items spanning every (bucket, w, k)
// group of the batch, then one launch for every query's top-k.
//
// Before it, each group's first stages ran as in a cascade run
// (cascade_prefix: envelopes, the stored bound of every pair, seeds, seed
// threshold).  A warp takes the next item from the queue and runs the rest of
// the cascade (Algorithm 3) on that chunk of candidates: the stored bound
// (the piecewise-sum bound or LB_Keogh, Sec. 7 and 9), LB_Keogh and
// LB_Improved's second sum (Sec. 8, the envelope form of k_lbi_filter), then
// the band DTW (Sec. 4) of the survivors, one warp per pair, each test
// against the query's live threshold b (1 + s).  A completed DTW lowers the
// threshold at once (atomicMin on its fp32 bits, through the group minima for
// k > 1) and is written back into the pair's matrix entry with the sign bit
// set, where the final top-k finds it.  Items are ordered group by group,
// heaviest group first, and within a group chunk by chunk, so that the CTAs
// in flight share a chunk's rows in L2.
#include "persist.cuh"

#include "dtw_kernels.cuh"

namespace dtwk {

constexpr int kPersistWarps = 8;
constexpr int kPersistSub = 1024;  // candidates a warp scans before testing them (its list capacity)

PersistShape persist_shape(int n, int w) {
    w = w < n - 1 ? w : n - 1;
    const int bw = 2 * w + 1;
    if (bw > 32 * 16) return PersistShape{0, 0};
    int g = 4;
    while (g * 16 < bw) g *= 2;
    for (int cl : {4, 8, 16})
        if (g * cl >= bw) return PersistShape{g, cl};
    return PersistShape{g, 16};
}

// DTW_p^p of one pair per group of G lanes (G = 4, 8, 16 or 32; 32 / G
// pairs per warp at once), band w with 2w + 1 <= G CL: lane l of a group
// owns band slots l CL .. l CL + CL - 1 (slot k of row i is column i - w + k)
// and computes row i at step 2i + l, its left neighbour's row i and its
// right neighbour's row i - 1 arriving by shuffles within the group one step
// old (the wavefront of k_dtw_wide).  x and yp (column 0 of the pair's query
// copy 0) and thr_bits (its live threshold) are the lane's group's; `live`
// says whether the group has a pair.  Every 8 steps the minimum of the last
// whole row, carried along the group's lanes, is compared with the live
// threshold; above it the pair is abandoned (every path crosses every row,
// and costs never decrease a path's value).  *res receives DTW^p or +INF
// (abandoned, or no pair), *rows the rows evaluated.
template <int CL, int P>
__device__ void group_dtw_band(int G, bool live, const float *__restrict__ x, const float *__restrict__ yp,
                               const uint32_t *thr_bits, int n, int w, float *res, int *rows) {
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1), gbase = lane - gl;
    const int top = 2 * w;
    const int lane_top = top / CL;
    const int lane_dead = (top + 1) / CL, c_dead = (top + 1) % CL;  // slot 2w + 1
    const int lane_diag = w / CL, c_diag = w % CL;                  // slot w: column i
    const int k0 = gl * CL;
    const bool computes = gl <= lane_dead;
    bool act = live;
    float D[CL], yw[CL];
#pragma unroll
    for (int t = 0; t < CL; ++t) {
        D[t] = (k0 + t == w) ? 0.0f : kInf;  // row -1: D(-1,-1) = 0
        yw[t] = (live && computes) ? __ldg(yp + (k0 + t - w)) : 0.0f;
    }
    float ex_first = D[0], ex_last = D[CL - 1], ex_min = kInf;
    int done_rows = n;
    const int steps = 2 * (n - 1) + lane_diag + 1;  // lane_diag computes row n - 1 at the last step
    for (int t = 0; t < steps; ++t) {
        if (!__any_sync(0xffffffffu, act)) break;
        float left = __shfl_up_sync(0xffffffffu, ex_last, 1, G);
        float up = __shfl_down_sync(0xffffffffu, ex_first, 1, G);
        float lmin = __shfl_up_sync(0xffffffffu, ex_min, 1, G);
        if (gl == 0) {
            left = kInf;
            lmin = kInf;
        }
        if (gl == G - 1) up = kInf;
        const int dd = t - gl;
        if (act && computes && dd >= 0 && !(dd & 1) && (dd >> 1) < n) {
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
                D[u] = dtw_cost<P>(xi - yw[u], min3f(D[u], above, below));
                mn = fminf(mn, D[u]);
            }
            if (gl == lane_dead) {
#pragma unroll
                for (int u = 0; u < CL; ++u) D[u] = sel_eq(u, c_dead, kInf, D[u]);  // outside the band
            }
            ex_first = D[0];
            ex_last = D[CL - 1];
            ex_min = (gl <= lane_top) ? fminf(mn, lmin) : lmin;
        }
        if ((t & 7) == 7 && t >= lane_top) {
            // the group's lane_top has completed a whole row; its running minimum covers it
            const float rowmin = __shfl_sync(0xffffffffu, ex_min, gbase + lane_top);
            const float thr = __shfl_sync(0xffffffffu, act ? load_threshold(thr_bits) : kInf, gbase);
            if (act && rowmin > thr) {
                act = false;
                live = false;
                done_rows = max(0, min(n, (t - lane_top) / 2 + 1));
            }
        }
    }
    float dv = kInf;
#pragma unroll
    for (int u = 0; u < CL; ++u) dv = sel_eq(u, c_diag, D[u], dv);
    dv = __shfl_sync(0xffffffffu, dv, gbase + lane_diag);
    *res = live ? dv : kInf;
    *rows = done_rows;
}

template <int P>
__device__ __forceinline__ void group_dtw_any(int cl, int G, bool live, const float *x, const float *yp,
                                              const uint32_t *thr_bits, int n, int w, float *res, int *rows) {
    switch (cl) {
        case 4: group_dtw_band<4, P>(G, live, x, yp, thr_bits, n, w, res, rows); break;
        case 8: group_dtw_band<8, P>(G, live, x, yp, thr_bits, n, w, res, rows); break;
        default: group_dtw_band<16, P>(G, live, x, yp, thr_bits, n, w, res, rows); break;
    }
}

// This lane's parts of LB_Keogh^p of (q, c) (a1, when `first`) and of
// LB_Improved's second sum in its envelope form (a2; see k_lbi_filter):
// lane l takes the 16-byte pieces l, l + 32, ... (g.vec) or the indices
// l, l + 32, ...
template <int P>
__device__ __forceinline__ void lane_pair_bounds(const PersistGroup &g, int q, int c, bool first, float &a1,
                                                 float &a2) {
    const int lane = threadIdx.x & 31;
    const int n = g.n;
    const int64_t oc = (int64_t)c * n, oq = (int64_t)q * n;
    const float *x = g.db + oc, *xu = g.XU + oc, *xl = g.XL + oc;
    const float *U = g.U + oq, *L = g.L + oq, *y = g.queries + oq, *ul = g.UL + oq, *lu = g.LU + oq;
    a1 = 0.0f;
    a2 = 0.0f;
    if (g.vec) {
        for (int i = 4 * lane; i < n; i += 128) {
            if (first) a1 = acc_dist4<P>(a1, ldg4(x + i), ldg4(L + i), ldg4(U + i));
            a2 = acc_dist4<P>(a2, ldg4(y + i), min4(ldg4(xl + i), ldg4(lu + i)), max4(ldg4(xu + i), ldg4(ul + i)));
        }
    } else {
        for (int i = lane; i < n; i += 32) {
            if (first) a1 = acc_dist<P>(a1, __ldg(x + i), __ldg(L + i), __ldg(U + i));
            a2 = acc_dist<P>(a2, __ldg(y + i), fminf(__ldg(xl + i), __ldg(lu + i)), fmaxf(__ldg(xu + i), __ldg(ul + i)));
        }
    }
}

template <int P>
__global__ void __launch_bounds__(kPersistWarps * 32, 2)
k_persist(const PersistGroup *__restrict__ groups, int G, int64_t total, unsigned long long *cursor) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *surv_c = reinterpret_cast<int32_t *>(smraw) + (size_t)wid * 2 * kPersistSub;
    float *surv_v = reinterpret_cast<float *>(surv_c + kPersistSub);
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(cursor, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if ((int64_t)it >= total) break;
        int lo = 0, hi = G - 1;  // the last group whose first item is <= it
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (groups[mid].item0 <= (int64_t)it) lo = mid;
            else hi = mid - 1;
        }
        const PersistGroup &g = groups[lo];
        const int64_t r = (int64_t)it - g.item0;
        const int chunk = (int)(r / g.Q), q = (int)(r - (int64_t)chunk * g.Q);
        const int n = g.n, w = g.w;
        const int c_begin = chunk * g.chunk, c_end = min(g.N, c_begin + g.chunk);
        float *lbrow = g.lb + (int64_t)q * g.N;
        const float *yp = g.qc.data + (int64_t)q * 4 * g.qc.ylen + g.qc.padl;
        uint32_t *bq = g.bsf + q;
        const float slack1 = 1.0f + g.slack;
        unsigned long long n_first = 0, n_keogh = 0, n_lbi = 0, n_skip = 0, n_comp = 0, n_ab = 0, n_rows = 0,
                           n_cells = 0;
        for (int s0 = c_begin; s0 < c_end; s0 += kPersistSub) {
            const int s1 = min(c_end, s0 + kPersistSub);
            // the stored bound against the live threshold; seeds hold NaN and never pass
            const float thr0 = __shfl_sync(0xffffffffu, load_threshold(bq), 0) * slack1;
            const float thr_m = g.summary ? thr0 * g.summary_scale : thr0;
            int cnt1 = 0;
            for (int base = s0; base < s1; base += 32) {
                const int c = base + lane;
                const float v = c < s1 ? __ldcs(lbrow + c) : kInf;
                const bool pass = c < s1 && v <= thr_m;
                const unsigned m = __ballot_sync(0xffffffffu, pass);
                if (pass) {
                    const int slot = cnt1 + __popc(m & ((1u << lane) - 1));
                    surv_c[slot] = c;
                    surv_v[slot] = v;
                }
                cnt1 += __popc(m);
            }
            __syncwarp();
            n_first += cnt1;
            // LB_Keogh (when the matrix held the piecewise-sum bound) and
            // LB_Improved, eight pairs at a time with one transposed
            // reduction (as in k_lbi_batch); the survivors stay in place
            int cnt2 = 0;
            for (int e0 = 0; e0 < cnt1; e0 += kLbiBatch) {
                float v[16];
#pragma unroll
                for (int u = 0; u < kLbiBatch; ++u) {
                    float a1 = 0.0f, a2 = 0.0f;
                    if (e0 + u < cnt1) lane_pair_bounds<P>(g, q, surv_c[e0 + u], g.summary != 0, a1, a2);
                    v[u] = a1;
                    v[u + 8] = a2;
                }
                const float r1 = warp_sum16_transposed(v);  // lane 2j: pair j's first sum
                const float r2 = __shfl_down_sync(0xffffffffu, r1, 16);  // lane 16 + 2j: its second
                const int j = lane >> 1;
                const bool decides = lane < 16 && !(lane & 1) && e0 + j < cnt1;
                const float thr = __shfl_sync(0xffffffffu, load_threshold(bq), 0) * slack1;
                const int c = decides ? surv_c[e0 + j] : 0;
                const float lbk = decides ? (g.summary ? r1 : surv_v[e0 + j]) : kInf;
                const float lbi = lbk + r2;
                const bool kpass = decides && lbk <= thr;
                const bool pass = kpass && lbi <= thr;
                n_keogh += __popc(__ballot_sync(0xffffffffu, kpass));
                const unsigned m = __ballot_sync(0xffffffffu, pass);
                __syncwarp();  // every decider has read its entry before the list is rewritten
                if (pass) {
                    const int at = cnt2 + __popc(m & ((1u << lane) - 1));
                    surv_c[at] = c;
                    surv_v[at] = lbi;
                }
                cnt2 += __popc(m);
                __syncwarp();
            }
            n_lbi += cnt2;
            // band DTW of the survivors, 32 / G pairs at a time (one per lane
            // group), each against the threshold as it is then
            const int G = g.dg, gl = lane & (G - 1), grp = lane / G;
            for (int e0 = 0; e0 < cnt2; e0 += 32 / G) {
                const int e = e0 + grp;
                bool live = e < cnt2;
                const int c = live ? surv_c[e] : 0;
                if (live) {
                    const float thr = load_threshold(bq) * slack1;
                    if (surv_v[e] > thr) {
                        live = false;
                        if (gl == 0) ++n_skip;
                    }
                }
                float d = kInf;
                int rows = 0;
                group_dtw_any<P>(g.cl, G, live, g.db + (int64_t)c * n, yp, bq, n, w, &d, &rows);
                if (live && gl == 0) {
                    ++n_comp;
                    n_rows += rows;
                    n_cells += (unsigned long long)band_cells(rows, n, w);
                    if (d < kInf) {
                        lbrow[c] = -d;  // a completed DTW^p: sign bit set
                        update_threshold(g.bsf, g.gmin, g.k, q, c % g.k, d);
                    } else {
                        ++n_ab;
                    }
                }
                __syncwarp();
            }
            __syncwarp();  // the lists are refilled by the next part of the chunk
        }
        // the DTW counters were kept by each group's first lane
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            n_skip += __shfl_xor_sync(0xffffffffu, n_skip, o);
            n_comp += __shfl_xor_sync(0xffffffffu, n_comp, o);
            n_ab += __shfl_xor_sync(0xffffffffu, n_ab, o);
            n_rows += __shfl_xor_sync(0xffffffffu, n_rows, o);
            n_cells += __shfl_xor_sync(0xffffffffu, n_cells, o);
        }
        if (lane == 0 && g.counters) {
            unsigned long long *cn = g.counters;
            if (g.summary) {
                if (n_first) atomicAdd(cn + CNT_SUMMARY_PASS, n_first);
            }
            if (n_keogh) atomicAdd(cn + CNT_KEOGH_PASS, n_keogh);
            if (n_lbi) atomicAdd(cn + CNT_LBI_PASS, n_lbi);
            if (n_skip) atomicAdd(cn + CNT_DTW_SKIP, n_skip);
            if (n_comp) atomicAdd(cn + CNT_DTW_COMPUTED, n_comp);
            if (n_ab) atomicAdd(cn + CNT_DTW_ABANDONED, n_ab);
            if (n_rows) atomicAdd(cn + CNT_DTW_ROWS, n_rows);
            if (n_cells) atomicAdd(cn + CNT_DTW_CELLS, n_cells);
        }
    }
}

__device__ __forceinline__ unsigned long long persist_key(float d, int c) {
    return ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)c;
}

// Top-k of one query of one group: the k smallest (distance, index) among
// its seeds and the completed DTWs in its matrix row, keeping only distances
// not above the final threshold (every true neighbour satisfies that).  The
// row's completed entries are first collected in shared memory (k rounds of
// a block-wide minimum then run over them); if they do not fit, the rounds
// run over the row itself.
constexpr int kFinalCap = 4096;

__global__ void __launch_bounds__(256) k_persist_finalize(const PersistGroup *__restrict__ groups, int G) {
    const int64_t gq = blockIdx.x;
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (groups[mid].qbase <= gq) lo = mid;
        else hi = mid - 1;
    }
    const PersistGroup &g = groups[lo];
    const int q = (int)(gq - g.qbase);
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const float bq = __uint_as_float(g.bsf[q]);
    const float *row = g.lb + (int64_t)q * g.N;
    __shared__ unsigned long long keys[kFinalCap];
    __shared__ int nkeys;
    __shared__ unsigned long long wmin[8];
    __shared__ unsigned long long sel;
    if (t == 0) nkeys = 0;
    __syncthreads();
    for (int c = t; c < g.N; c += blockDim.x) {
        const uint32_t u = __float_as_uint(row[c]);
        if (u & 0x80000000u) {
            const float d = __uint_as_float(u & 0x7fffffffu);
            if (d <= bq) {
                const int at = atomicAdd(&nkeys, 1);
                if (at < kFinalCap) keys[at] = persist_key(d, c);
            }
        }
    }
    __syncthreads();
    const bool in_smem = nkeys <= kFinalCap;
    unsigned long long last = 0;
    bool first = true;
    for (int r = 0; r < g.k; ++r) {
        unsigned long long m = ~0ull;
        for (int s = t; s < g.S; s += blockDim.x) {
            const Pair pr = g.seed_pairs[(int64_t)s * g.Q + q];
            const float d = g.seed_res[(int64_t)s * g.Q + q];
            if (pr.c >= 0 && d < kInf && d <= bq) {
                const unsigned long long v = persist_key(d, pr.c);
                if ((first || v > last) && v < m) m = v;
            }
        }
        if (in_smem) {
            for (int e = t; e < nkeys; e += blockDim.x) {
                const unsigned long long v = keys[e];
                if ((first || v > last) && v < m) m = v;
            }
        } else {
            for (int c = t; c < g.N; c += blockDim.x) {
                const uint32_t u = __float_as_uint(row[c]);
                if (!(u & 0x80000000u)) continue;
                const float d = __uint_as_float(u & 0x7fffffffu);
                if (d > bq) continue;
                const unsigned long long v = persist_key(d, c);
                if ((first || v > last) && v < m) m = v;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, m, o);
            m = other < m ? other : m;
        }
        if (lane == 0) wmin[wid] = m;
        __syncthreads();
        if (t == 0) {
            unsigned long long best = wmin[0];
            for (int v = 1; v < (int)(blockDim.x >> 5); ++v) best = wmin[v] < best ? wmin[v] : best;
            sel = best;
            const int64_t o = (int64_t)q * g.k + r;
            if (best == ~0ull) {
                g.out_idx[o] = -1;
                g.out_dist[o] = kInf;
            } else {
                g.out_idx[o] = (int64_t)(best & 0xffffffffull);
                g.out_dist[o] = root_p(__uint_as_float((uint32_t)(best >> 32)), g.p);
            }
        }
        __syncthreads();
        last = sel;
        first = false;
        if (last == ~0ull) {
            for (int rr = r + 1 + t; rr < g.k; rr += blockDim.x) {
                g.out_idx[(int64_t)q * g.k + rr] = -1;
                g.out_dist[(int64_t)q * g.k + rr] = kInf;
            }
            break;
        }
        __syncthreads();
    }
}

cudaError_t launch_persistent(const PersistGroup *groups, int G, int64_t total_items, int64_t total_queries,
                              int p, unsigned long long *cursor, cudaStream_t s) {
    if (G <= 0) return cudaSuccess;
    if (total_items > 0) {
        auto kern = p == 1 ? k_persist<1> : k_persist<2>;
        const size_t smem = (size_t)kPersistWarps * kPersistSub * 8;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPersistWarps * 32, smem);
        if (per_sm < 1) per_sm = 1;
        int64_t blocks = (int64_t)per_sm * device_sm_count();
        const int64_t need = (total_items + kPersistWarps - 1) / kPersistWarps;
        if (blocks > need) blocks = need;
        kern<<<(int)blocks, kPersistWarps * 32, smem, s>>>(groups, G, total_items, cursor);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (total_queries > 0) k_persist_finalize<<<(unsigned)total_queries, 256, 0, s>>>(groups, G);
    return cudaGetLastError();
}

}  // namespace dtwk

// Best-so-far linking of the cascade (Algorithms 2 and 3, generalised to k
// neighbours): seed selection, the seed threshold, and the final ordered
// top-k.  The threshold b of a query is its current k-th best DTW_p^p (fp32
// bits, so that atomicMin orders it); candidates are compared by
// (distance, index), so ties go to the lower index as in a sequential scan
// with strict "<" tests.
#include "common.cuh"

namespace dtwk {

constexpr int kSeedMax = 32;

__device__ __forceinline__ unsigned long long pack_key(float d, int c) {
    return ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)c;
}

// ---------------------------------------------------------------------------
// Seeds: per query, the S smallest of the per-tile LB_Keogh minima (each the
// smallest (bound, index) among 128 consecutive candidates), or for small
// databases (N <= 8192) the S smallest bounds overall.  Their exact DTW
// is computed first so that the threshold is close to its final value before
// the bulk of the candidates is filtered; this is the GPU counterpart of
// visiting candidates in order of their lower bound.  One warp per query:
// each lane keeps a sorted list of its kSeedMax best keys, then S rounds of a
// warp minimum pop the global best (no block barriers).  The seed of rank s
// of query q is stored at s * Q + q, so the k best-bounded seeds of every
// query come first.  Also resets the query's thresholds to +INF.
// ---------------------------------------------------------------------------
constexpr int kSeedWarps = 4;

__global__ void __launch_bounds__(kSeedWarps * 32) k_seed_select(CascadeBufs b) {
    const int q = blockIdx.x * kSeedWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (q >= b.Q) return;
    if (lane == 0) b.bsf[q] = 0x7f800000u;
    for (int g = lane; g < b.k; g += 32) b.gmin[(int64_t)q * b.k + g] = 0x7f800000u;
    unsigned long long key[kSeedMax];
#pragma unroll
    for (int s = 0; s < kSeedMax; ++s) key[s] = ~0ull;
    // small databases: scan every bound (the tiles may be fewer than S)
    const bool full = b.N <= 8192;
    const int cnt = full ? b.N : b.ntiles;
    const float *lbrow = b.lb + (int64_t)q * b.N;
    const unsigned long long *row = b.tile_min + (int64_t)q * b.ntiles;
    for (int c = lane; c < cnt; c += 32) {
        unsigned long long v = full ? pack_key(lbrow[c], c) : row[c];
        if (v < key[kSeedMax - 1]) {
            // insertion into the sorted list
#pragma unroll
            for (int s = kSeedMax - 1; s > 0; --s) {
                unsigned long long prev = key[s - 1];
                bool shift = v < prev;
                key[s] = shift ? prev : (v < key[s] ? v : key[s]);
            }
            key[0] = v < key[0] ? v : key[0];
        }
    }
    // every lane has read its bounds before the seeds' entries become NaN
    __syncwarp();
    for (int s = 0; s < b.S; ++s) {
        unsigned long long m = key[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long other = __shfl_xor_sync(0xffffffffu, m, o);
            m = other < m ? other : m;
        }
        if (lane == 0) {
            const int c = (m == ~0ull) ? -1 : (int)(unsigned)(m & 0xffffffffull);
            b.seed_pairs[(int64_t)s * b.Q + q] = Pair{q, c};
            b.seed_res[(int64_t)s * b.Q + q] = kInf;
            // the seed's matrix entry becomes NaN, which no bound test passes:
            // the filter then skips seeds without looking them up
            if (c >= 0) b.lb[(int64_t)q * b.N + c] = __int_as_float(0x7fc00000);
        }
        if (key[0] == m && m != ~0ull) {
            // pop: only the owner holds this (unique) key
#pragma unroll
            for (int u = 0; u + 1 < kSeedMax; ++u) key[u] = key[u + 1];
            key[kSeedMax - 1] = ~0ull;
        }
    }
}

cudaError_t launch_seed_select(const CascadeBufs &b, cudaStream_t s) {
    if (b.Q <= 0) return cudaSuccess;
    k_seed_select<<<(b.Q + kSeedWarps - 1) / kSeedWarps, kSeedWarps * 32, 0, s>>>(b);
    return cudaGetLastError();
}

// After the seeds' DTW: b = k-th smallest seed distance (one warp per query).
__global__ void k_seed_kth(CascadeBufs b) {
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (q >= b.Q) return;
    unsigned long long mine = ~0ull;
    if (lane < b.S) {
        Pair pr = b.seed_pairs[(int64_t)lane * b.Q + q];
        float d = b.seed_res[(int64_t)lane * b.Q + q];
        if (pr.c >= 0 && d < kInf) mine = pack_key(d, pr.c);
    }
    int rank = 0;
    for (int o = 0; o < 32; ++o) {
        unsigned long long other = __shfl_sync(0xffffffffu, mine, o);
        rank += (other < mine) ? 1 : 0;
    }
    if (mine != ~0ull && rank == b.k - 1) atomicMin(b.bsf + q, (uint32_t)(mine >> 32));
}

cudaError_t launch_seed_kth(const CascadeBufs &b, cudaStream_t s) {
    if (b.Q <= 0 || b.S < b.k) return cudaSuccess;
    const int per = 4;
    k_seed_kth<<<(b.Q + per - 1) / per, 32 * per, 0, s>>>(b);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Final top-k per query: the k smallest (distance, index) keys among the
// seeds and the listed pairs whose DTW completed, keeping only distances not
// above the final threshold (every true neighbour satisfies that).  k rounds
// of a block-wide minimum over keys greater than the previous round's key.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_finalize(CascadeBufs b) {
    const int q = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const float bq = __uint_as_float(b.bsf[q]);
    __shared__ unsigned long long wmin[8];
    __shared__ unsigned long long sel;
    unsigned long long last = 0;
    bool first = true;
    for (int r = 0; r < b.k; ++r) {
        unsigned long long m = ~0ull;
        for (int s = t; s < b.S; s += blockDim.x) {
            Pair pr = b.seed_pairs[(int64_t)s * b.Q + q];
            float d = b.seed_res[(int64_t)s * b.Q + q];
            if (pr.c >= 0 && d < kInf && d <= bq) {
                unsigned long long v = pack_key(d, pr.c);
                if ((first || v > last) && v < m) m = v;
            }
        }
        if (b.nseg > 0) {
            const int cnt = b.qcount[q];
            const int lead = b.order_first > 0 ? (cnt < b.order_first ? cnt : b.order_first) : cnt;
            const int64_t base = b.qstart[q];
            const int64_t base_b = b.order_first > 0 ? b.qstart_b[q] - lead : 0;
            for (int e = t; e < cnt; e += blockDim.x) {
                const int64_t at = e < lead ? base + e : base_b + e;
                float d = b.pair_res[at];
                if (d < kInf && d <= bq) {
                    unsigned long long v = pack_key(d, b.pairs[at].c);
                    if ((first || v > last) && v < m) m = v;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long other = __shfl_xor_sync(0xffffffffu, m, o);
            m = other < m ? other : m;
        }
        if (lane == 0) wmin[wid] = m;
        __syncthreads();
        if (t == 0) {
            unsigned long long best = wmin[0];
            for (int v = 1; v < (int)(blockDim.x >> 5); ++v) best = wmin[v] < best ? wmin[v] : best;
            sel = best;
            int64_t o = (int64_t)q * b.k + r;
            if (best == ~0ull) {
                b.out_idx[o] = -1;
                b.out_dist[o] = kInf;
            } else {
                b.out_idx[o] = (int64_t)(best & 0xffffffffull);
                b.out_dist[o] = root_p(__uint_as_float((uint32_t)(best >> 32)), b.p);
            }
        }
        __syncthreads();
        last = sel;
        first = false;
        if (last == ~0ull) {
            // nothing left: pad the remaining ranks
            for (int rr = r + 1 + t; rr < b.k; rr += blockDim.x) {
                b.out_idx[(int64_t)q * b.k + rr] = -1;
                b.out_dist[(int64_t)q * b.k + rr] = kInf;
            }
            break;
        }
        __syncthreads();
    }
}

cudaError_t launch_finalize(const CascadeBufs &b, cudaStream_t s) {
    if (b.Q <= 0) return cudaSuccess;
    k_finalize<<<b.Q, 256, 0, s>>>(b);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Thresholds shared between the shards of a candidate-sharded search: each
// query's threshold lowered to an outside value (NaN and negative values are
// ignored), and/or copied out.  Costs are non-negative, so the fp32 bits of
// the thresholds order like their values.
// ---------------------------------------------------------------------------
__global__ void k_threshold_io(uint32_t *bsf, int Q, int has_db, const float *thr_in, float *thr_out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    uint32_t v = has_db ? bsf[q] : 0x7f800000u;
    if (thr_in) {
        const float t = thr_in[q] + 0.0f;  // -0 -> +0
        if (t >= 0.0f) {
            const uint32_t tb = __float_as_uint(t);
            v = tb < v ? tb : v;
        }
    }
    if (has_db) bsf[q] = v;
    if (thr_out) thr_out[q] = __uint_as_float(v);
}

cudaError_t launch_threshold_io(uint32_t *bsf, int Q, bool has_db, const float *thr_in, float *thr_out,
                                cudaStream_t s) {
    if (Q <= 0 || (!thr_in && !thr_out)) return cudaSuccess;
    k_threshold_io<<<(Q + 255) / 256, 256, 0, s>>>(bsf, Q, has_db ? 1 : 0, thr_in, thr_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Merge of per-shard top-k lists (candidate sharding): one warp per query
// takes the k smallest (distance, index) keys among the R lists of k_in
// entries ([R][Q][k_in], global indices, -1 / +INF empty), k rounds of a
// warp minimum over the keys above the previous round's.
// ---------------------------------------------------------------------------
__global__ void k_merge_topk(const int64_t *idx, const float *dist, int R, int Q, int k_in, int k,
                             int64_t *out_idx, float *out_dist) {
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (q >= Q) return;
    const int m = R * k_in;
    unsigned long long last = 0;
    bool first = true;
    for (int r = 0; r < k; ++r) {
        unsigned long long best = ~0ull;
        for (int e = lane; e < m; e += 32) {
            const int sh = e / k_in, t = e - sh * k_in;
            const int64_t at = ((int64_t)sh * Q + q) * k_in + t;
            const int64_t c = idx[at];
            const float d = dist[at];
            if (c < 0 || !(d < kInf)) continue;
            const unsigned long long v = pack_key(d + 0.0f, (int)c);
            if ((first || v > last) && v < best) best = v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
            best = other < best ? other : best;
        }
        const int64_t o = (int64_t)q * k + r;
        if (lane == 0) {
            out_idx[o] = best == ~0ull ? -1 : (int64_t)(best & 0xffffffffull);
            out_dist[o] = best == ~0ull ? kInf : __uint_as_float((uint32_t)(best >> 32));
        }
        last = best;
        first = false;
    }
}

cudaError_t launch_merge_topk(const int64_t *idx, const float *dist, int R, int Q, int k_in, int k,
                              int64_t *out_idx, float *out_dist, cudaStream_t s) {
    if (Q <= 0) return cudaSuccess;
    const int per = 4;
    k_merge_topk<<<(Q + per - 1) / per, 32 * per, 0, s>>>(idx, dist, R, Q, k_in, k, out_idx, out_dist);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Group the filter's survivors by query (a counting sort): exclusive scans of
// the per-query counts give each query its output ranges, and one CTA per
// query moves its sub-segments there.  The DTW stage then sees runs of pairs
// that share a query (warp-uniform band-window loads).
//
// With order_first = F > 0 the CTA also orders its query's pairs by bound:
// bin = floor(256 * bound / threshold), a histogram and its scan give each
// pair a rank, and rank r goes to the leading region (r < F) or to the
// query's range after it.  The leading region holds every query's F
// lowest-bound pairs, so the DTW stage computes the likeliest neighbours of
// all queries before anything else.
// ---------------------------------------------------------------------------
constexpr int kOrderBins = 256;

// Exclusive scan over Q of f(cnt[i]) into out[i] + base, one CTA; returns the total.
template <typename F>
__device__ int32_t block_scan_counts(const int32_t *__restrict__ cnt, int32_t *__restrict__ out, int Q, int32_t base,
                                     F f) {
    __shared__ int32_t wsum[32];
    __shared__ int32_t carry;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0) carry = base;
    __syncthreads();
    for (int b0 = 0; b0 < Q; b0 += blockDim.x) {
        const int i = b0 + t;
        const int v = i < Q ? f(cnt[i]) : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int s = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;  // inclusive over warps
        }
        __syncthreads();
        const int before = (wid > 0 ? wsum[wid - 1] : 0) + carry;
        if (i < Q) out[i] = before + x - v;
        __syncthreads();
        if (t == blockDim.x - 1) carry = before + x;
        __syncthreads();
    }
    const int32_t total = carry;
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(1024) k_qscan(const int32_t *__restrict__ cnt, int32_t *__restrict__ start,
                                                int32_t *__restrict__ start_b, int Q, int first,
                                                unsigned long long *total, unsigned long long *lead_total) {
    if (first <= 0) {
        const int32_t all = block_scan_counts(cnt, start, Q, 0, [](int32_t c) { return c; });
        if (threadIdx.x == 0 && total) *total = (unsigned long long)all;
        if (threadIdx.x == 0 && lead_total) *lead_total = 0;
        return;
    }
    const int32_t lead = block_scan_counts(cnt, start, Q, 0, [first](int32_t c) { return c < first ? c : first; });
    const int32_t all =
        block_scan_counts(cnt, start_b, Q, lead, [first](int32_t c) { return c > first ? c - first : 0; });
    if (threadIdx.x == 0 && total) *total = (unsigned long long)all;
    if (threadIdx.x == 0 && lead_total) *lead_total = (unsigned long long)lead;
}

__device__ __forceinline__ int order_bin(float bound, float scale) {
    const float r = bound * scale;
    return r < (float)(kOrderBins - 1) ? (int)r : kOrderBins - 1;  // bound >= 0
}

__global__ void __launch_bounds__(256) k_gather(CascadeBufs b) {
    const int q = blockIdx.x;
    const int t = threadIdx.x;
    __shared__ int32_t offs[256];
    __shared__ int32_t carry;
    const int64_t out0 = b.qstart[q];
    const int F = b.order_first;
    if (F > 0) {
        __shared__ int32_t hist[kOrderBins];
        const int64_t outb = b.qstart_b[q];
        const int cq = b.qcount[q];
        const int lead = cq < F ? cq : F;
        const float thr = __uint_as_float(b.bsf[q]);
        // bins relative to the threshold the filter used; without a finite
        // positive threshold every pair shares bin 0
        const float scale = (thr > 0.0f && thr < kInf) ? (float)kOrderBins / thr : 0.0f;
        for (int i = t; i < kOrderBins; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int sg = t; sg < b.nseg; sg += blockDim.x) {
            const int c = b.seg_count[(int64_t)q * b.nseg + sg];
            const int64_t src = b.seg_start[(int64_t)q * b.nseg + sg];
            for (int e = 0; e < c; ++e) atomicAdd(&hist[order_bin(b.lbi_u[src + e], scale)], 1);
        }
        __syncthreads();
        // exclusive scan of the histogram (kOrderBins == blockDim.x)
        const int h = hist[t];
        offs[t] = h;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const int v = t >= o ? offs[t - o] : 0;
            __syncthreads();
            offs[t] += v;
            __syncthreads();
        }
        hist[t] = offs[t] - h;
        __syncthreads();
        for (int sg = t; sg < b.nseg; sg += blockDim.x) {
            const int c = b.seg_count[(int64_t)q * b.nseg + sg];
            const int64_t src = b.seg_start[(int64_t)q * b.nseg + sg];
            for (int e = 0; e < c; ++e) {
                const float lb = b.lbi_u[src + e];
                const int r = atomicAdd(&hist[order_bin(lb, scale)], 1);
                const int64_t dst = r < lead ? out0 + r : outb + (r - lead);
                const Pair pr = b.pairs_u[src + e];
                b.pairs[dst] = pr;
                b.pair_lbi[dst] = lb;
                b.pair_res[dst] = b.lb[(int64_t)q * b.N + pr.c];  // LB_Keogh^p (see CascadeBufs)
            }
        }
        return;
    }
    if (t == 0) carry = 0;
    __syncthreads();
    for (int s0 = 0; s0 < b.nseg; s0 += blockDim.x) {
        const int sg = s0 + t;
        const int c = sg < b.nseg ? b.seg_count[(int64_t)q * b.nseg + sg] : 0;
        // block exclusive scan of the sub-segment counts (simple, nseg is small)
        offs[t] = c;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const int v = t >= o ? offs[t - o] : 0;
            __syncthreads();
            offs[t] += v;
            __syncthreads();
        }
        const int excl = offs[t] - c + carry;
        __syncthreads();
        if (t == blockDim.x - 1) carry += offs[t];
        // copy this sub-segment (one thread per sub-segment; they are short)
        if (sg < b.nseg && c > 0) {
            const int64_t src = b.seg_start[(int64_t)q * b.nseg + sg];
            for (int e = 0; e < c; ++e) {
                const Pair pr = b.pairs_u[src + e];
                b.pairs[out0 + excl + e] = pr;
                b.pair_lbi[out0 + excl + e] = b.lbi_u[src + e];
                b.pair_res[out0 + excl + e] = b.lb[(int64_t)q * b.N + pr.c];  // LB_Keogh^p
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_group_by_query(const CascadeBufs &b, cudaStream_t s) {
    if (b.Q <= 0 || b.nseg <= 0) return cudaSuccess;
    static_assert(kOrderBins == 256, "k_gather scans the histogram with one thread per bin");
    k_qscan<<<1, 1024, 0, s>>>(b.qcount, b.qstart, b.qstart_b, b.Q, b.order_first, b.pair_total, b.lead_total);
    k_gather<<<b.Q, 256, 0, s>>>(b);
    return cudaGetLastError();
}

// Shifted, +INF-padded query copies only (no envelope), for dtw_band.
__global__ void k_query_copies(const float *__restrict__ y, int64_t count, int n, float *copies,
                               int padl, int ylen) {
    const int64_t total = count * 4 * (int64_t)ylen;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = o / (4 * (int64_t)ylen);
        int rem = (int)(o - row * 4 * (int64_t)ylen);
        int r = rem / ylen, tt = rem - r * ylen;
        int j = tt + r - padl;
        copies[o] = (j >= 0 && j < n) ? y[row * n + j] : kInf;
    }
}

cudaError_t launch_query_copies(const float *y, int64_t count, int n, QueryCopies qc, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    int64_t total = count * 4 * (int64_t)qc.ylen;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)device_sm_count() * 16);
    k_query_copies<<<blocks, 256, 0, s>>>(y, count, n, qc.data, qc.padl, qc.ylen);
    return cudaGetLastError();
}

}  // namespace dtwk

// LB_Keogh (Sec. 7) and LB_Improved (Sec. 8) kernels.
//
//   LB_Keogh_p(x, y)^p    = sum_i d(x_i, [L(y)_i, U(y)_i])^p            (Eq. 1)
//   LB_Improved_p(x, y)^p = LB_Keogh_p(x, y)^p + LB_Keogh_p(y, H(x, y))^p
//
// where H(x, y) clamps x into the envelope of y.  All sums are fp32 in power
// space; the root is taken only where a bound is returned to the caller.
#include "common.cuh"

namespace dtwk {

// ---------------------------------------------------------------------------
// One query against N candidates: a streaming, HBM-bound pass.  The query
// envelope sits in shared memory; each warp owns one candidate at a time and
// reads it with coalesced 128-bit loads (scalar loads when rows are not
// 16-byte aligned), then reduces with shuffles.
// ---------------------------------------------------------------------------
template <int P, bool VEC>
__global__ void __launch_bounds__(256)
k_lbk_single(const float *__restrict__ cand, int64_t N, const float *__restrict__ U,
             const float *__restrict__ L, int n, float *__restrict__ out) {
    extern __shared__ float sm[];
    float *su = sm, *sl = sm + n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        su[i] = U[i];
        sl[i] = L[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < N; c += warps) {
        const float *x = cand + c * n;
        float acc = 0.0f;
        if (VEC) {
            const float4 *x4 = reinterpret_cast<const float4 *>(x);
            for (int v = lane; v < (n >> 2); v += 32) {
                float4 a = __ldcs(x4 + v);  // streamed once
                int i = v << 2;
                acc = acc_dist<P>(acc, a.x, sl[i], su[i]);
                acc = acc_dist<P>(acc, a.y, sl[i + 1], su[i + 1]);
                acc = acc_dist<P>(acc, a.z, sl[i + 2], su[i + 2]);
                acc = acc_dist<P>(acc, a.w, sl[i + 3], su[i + 3]);
            }
        } else {
            for (int i = lane; i < n; i += 32) acc = acc_dist<P>(acc, __ldcs(x + i), sl[i], su[i]);
        }
        acc = warp_sum(acc);
        if (lane == 0) out[c] = root_p(acc, P);
    }
}

cudaError_t launch_lbk_single(const float *cand, int64_t N, const float *U, const float *L, int n,
                              int p, float *out, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    bool vec = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(cand) & 15) == 0);
    int blocks = (int)std::min<int64_t>((N + 7) / 8, (int64_t)device_sm_count() * 8);
    size_t smem = 2 * (size_t)n * sizeof(float);
    if (p == 1) {
        if (vec) k_lbk_single<1, true><<<blocks, 256, smem, s>>>(cand, N, U, L, n, out);
        else k_lbk_single<1, false><<<blocks, 256, smem, s>>>(cand, N, U, L, n, out);
    } else {
        if (vec) k_lbk_single<2, true><<<blocks, 256, smem, s>>>(cand, N, U, L, n, out);
        else k_lbk_single<2, false><<<blocks, 256, smem, s>>>(cand, N, U, L, n, out);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// All pairs: lb[q][c] = LB_Keogh_p(db[c], queries[q])^p for a tile of
// TQ = 32 queries x TC = 128 candidates per CTA.  Element chunks of KC = 32
// are staged in shared memory with cp.async (double-buffered); warp v owns
// queries 4v..4v+3 and lane l owns candidates l, l+32, l+64, l+96, so the
// candidate reads are conflict-free 128-bit loads and the envelope reads are
// warp-wide broadcasts.  Out-of-range elements and candidates are
// zero-filled: x = U = L = 0 contributes nothing.  Each thread keeps 16
// accumulators (4 queries x 4 candidates), summed per chunk and then added to
// the running total.  Each CTA also writes, per query, the smallest
// (bound, index) key over its 128 candidates, from which the seeds are drawn.
// ---------------------------------------------------------------------------
constexpr int TQ = 32, TC = 128, KC = 32, XS = KC + 4;  // XS: padded row stride

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool pred) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    int sz = pred ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, bool pred) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    int sz = pred ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

struct TileSmem {
    float x[2][TC * XS];
    float u[2][TQ * KC];
    float l[2][TQ * KC];
};

template <bool VEC>
__device__ __forceinline__ void tile_load(TileSmem &sm, int buf, const float *db, int N,
                                          const float *U, const float *L, int Q, int n, int c0,
                                          int q0, int k0) {
    const int t = threadIdx.x;
    if (VEC) {
        // candidates: TC rows x KC floats = 1024 float4, 4 per thread
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int f = t + 256 * s;
            int r = f >> 3, g = f & 7;
            int c = c0 + r, k = k0 + 4 * g;
            bool ok = (c < N) && (k < n);
            const float *src = ok ? db + (int64_t)c * n + k : db;
            cp_async16(&sm.x[buf][r * XS + 4 * g], src, ok);
        }
        // envelopes: TQ rows x KC floats, U and L: 2 x 256 float4, 1 each per thread
        {
            int r = t >> 3, g = t & 7;
            int q = q0 + r, k = k0 + 4 * g;
            bool ok = (q < Q) && (k < n);
            int64_t off = ok ? (int64_t)q * n + k : 0;
            cp_async16(&sm.u[buf][r * KC + 4 * g], U + off, ok);
            cp_async16(&sm.l[buf][r * KC + 4 * g], L + off, ok);
        }
    } else {
        for (int f = t; f < TC * KC; f += 256) {
            int r = f / KC, kk = f % KC;
            int c = c0 + r, k = k0 + kk;
            bool ok = (c < N) && (k < n);
            cp_async4(&sm.x[buf][r * XS + kk], ok ? db + (int64_t)c * n + k : db, ok);
        }
        for (int f = t; f < TQ * KC; f += 256) {
            int r = f / KC, kk = f % KC;
            int q = q0 + r, k = k0 + kk;
            bool ok = (q < Q) && (k < n);
            int64_t off = ok ? (int64_t)q * n + k : 0;
            cp_async4(&sm.u[buf][r * KC + kk], U + off, ok);
            cp_async4(&sm.l[buf][r * KC + kk], L + off, ok);
        }
    }
    cp_async_commit();
}

template <int P, bool VEC>
__global__ void __launch_bounds__(256)
k_lbk_tile(const float *__restrict__ db, int N, const float *__restrict__ U,
           const float *__restrict__ L, int Q, int n, float *__restrict__ lb,
           unsigned long long *__restrict__ tile_min) {
    extern __shared__ __align__(16) unsigned char smraw[];
    TileSmem &sm = *reinterpret_cast<TileSmem *>(smraw);
    const int c0 = blockIdx.x * TC;
    const int q0 = blockIdx.y * TQ;
    const int lane = threadIdx.x & 31;
    const int wq = (threadIdx.x >> 5) * 4;  // first query row of this warp in the tile
    float tot[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) tot[a][b] = 0.0f;

    const int nchunks = (n + KC - 1) / KC;
    tile_load<VEC>(sm, 0, db, N, U, L, Q, n, c0, q0, 0);
    for (int ch = 0; ch < nchunks; ++ch) {
        const int buf = ch & 1;
        if (ch + 1 < nchunks) {
            tile_load<VEC>(sm, buf ^ 1, db, N, U, L, Q, n, c0, q0, (ch + 1) * KC);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
        const float *xs = sm.x[buf];
        const float *us = sm.u[buf];
        const float *ls = sm.l[buf];
#pragma unroll 2
        for (int k = 0; k < KC; k += 4) {
            float4 xv[4], uv[4], lv[4];
#pragma unroll
            for (int b = 0; b < 4; ++b)
                xv[b] = *reinterpret_cast<const float4 *>(&xs[(lane + 32 * b) * XS + k]);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                uv[a] = *reinterpret_cast<const float4 *>(&us[(wq + a) * KC + k]);
                lv[a] = *reinterpret_cast<const float4 *>(&ls[(wq + a) * KC + k]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    float s = acc[a][b];
                    s = acc_dist<P>(s, xv[b].x, lv[a].x, uv[a].x);
                    s = acc_dist<P>(s, xv[b].y, lv[a].y, uv[a].y);
                    s = acc_dist<P>(s, xv[b].z, lv[a].z, uv[a].z);
                    s = acc_dist<P>(s, xv[b].w, lv[a].w, uv[a].w);
                    acc[a][b] = s;
                }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) tot[a][b] += acc[a][b];
        __syncthreads();  // buffer `buf` is refilled in the next iteration
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int q = q0 + wq + a;
        unsigned long long key = ~0ull;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int c = c0 + lane + 32 * b;
            if (c < N && q < Q) {
                lb[(int64_t)q * N + c] = tot[a][b];
                const unsigned long long v = ((unsigned long long)__float_as_uint(tot[a][b]) << 32) | (unsigned)c;
                key = v < key ? v : key;
            }
        }
        // smallest (bound, index) of this query over the tile's 128 candidates
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
            key = other < key ? other : key;
        }
        if (lane == 0 && q < Q && tile_min) tile_min[(int64_t)q * gridDim.x + blockIdx.x] = key;
    }
}

int lbk_tiles(int N) { return (N + TC - 1) / TC; }

cudaError_t launch_lbk_tile(const float *db, int N, const float *U, const float *L, int Q, int n,
                            int p, float *lb, unsigned long long *tile_min, cudaStream_t s) {
    if (N <= 0 || Q <= 0) return cudaSuccess;
    bool vec = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(db) & 15) == 0) &&
               ((reinterpret_cast<uintptr_t>(U) & 15) == 0) &&
               ((reinterpret_cast<uintptr_t>(L) & 15) == 0);
    dim3 grid((N + TC - 1) / TC, (Q + TQ - 1) / TQ);
    size_t smem = sizeof(TileSmem);
    auto set = [&](const void *f) {
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    };
    if (p == 1) {
        if (vec) { set((const void *)k_lbk_tile<1, true>); k_lbk_tile<1, true><<<grid, 256, smem, s>>>(db, N, U, L, Q, n, lb, tile_min); }
        else { set((const void *)k_lbk_tile<1, false>); k_lbk_tile<1, false><<<grid, 256, smem, s>>>(db, N, U, L, Q, n, lb, tile_min); }
    } else {
        if (vec) { set((const void *)k_lbk_tile<2, true>); k_lbk_tile<2, true><<<grid, 256, smem, s>>>(db, N, U, L, Q, n, lb, tile_min); }
        else { set((const void *)k_lbk_tile<2, false>); k_lbk_tile<2, false><<<grid, 256, smem, s>>>(db, N, U, L, Q, n, lb, tile_min); }
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// LB_Improved of one pair by one warp (Sec. 8).  Lane l owns the indices
// i = l + 32 t.  The projection h = H(x, y) is written to the warp's shared
// scratch, its envelope with the same w is built by doubling (as in the
// envelope kernel), then the distance from y to that envelope is summed.
// scratch: 4n floats per warp.  Returns LB_Improved^p on every lane and the
// first-pass sum LB_Keogh^p in *lbk.
// ---------------------------------------------------------------------------
template <int P>
__device__ float warp_lb_improved(const float *__restrict__ x, const float *__restrict__ y,
                                  const float *__restrict__ U, const float *__restrict__ L, int n,
                                  int w, float *scratch, float *lbk) {
    const int lane = threadIdx.x & 31;
    float *ax = scratch, *an = scratch + n, *bx = scratch + 2 * n, *bn = scratch + 3 * n;
    float acc1 = 0.0f;
    for (int i = lane; i < n; i += 32) {
        float xv = __ldg(x + i);
        float u = __ldg(U + i), l = __ldg(L + i);
        float h = fminf(fmaxf(xv, l), u);  // Eq. 1 (L <= U)
        float d = fabsf(xv - h);
        acc1 = (P == 1) ? acc1 + d : fmaf(d, d, acc1);
        ax[i] = h;
        an[i] = h;
    }
    __syncwarp();
    const int len_max = min(2 * w + 1, n);
    const int kmax = 31 - __clz(len_max);
    for (int j = 1; j <= kmax; ++j) {
        const int hh = 1 << (j - 1);
        for (int i = lane; i < n; i += 32) {
            int i2 = min(i + hh, n - 1);
            bx[i] = fmaxf(ax[i], ax[i2]);
            bn[i] = fminf(an[i], an[i2]);
        }
        __syncwarp();
        float *t;
        t = ax; ax = bx; bx = t;
        t = an; an = bn; bn = t;
    }
    float acc2 = 0.0f;
    for (int i = lane; i < n; i += 32) {
        int a = max(0, i - w), b = min(n - 1, i + w);
        int k = 31 - __clz(b - a + 1);
        const float *tx = (k == kmax) ? ax : bx;
        const float *tn = (k == kmax) ? an : bn;
        int b2 = b - (1 << k) + 1;
        float uu = fmaxf(tx[a], tx[b2]);
        float ll = fminf(tn[a], tn[b2]);
        acc2 = acc_dist<P>(acc2, __ldg(y + i), ll, uu);
    }
    __syncwarp();  // scratch is reused by the next pair
    acc1 = warp_sum(acc1);
    acc2 = warp_sum(acc2);
    *lbk = acc1;
    return acc1 + acc2;
}

// All N candidates against one query, no threshold.
template <int P>
__global__ void __launch_bounds__(128)
k_lbi_single(const float *__restrict__ cand, int64_t N, const float *__restrict__ q,
             const float *__restrict__ U, const float *__restrict__ L, int n, int w,
             float *__restrict__ out) {
    extern __shared__ float sm[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *scratch = sm + (size_t)wid * 4 * n;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid; c < N; c += warps) {
        float lbk;
        float v = warp_lb_improved<P>(cand + c * n, q, U, L, n, w, scratch, &lbk);
        if (lane == 0) out[c] = root_p(v, P);
    }
}

cudaError_t launch_lbi_single(const float *cand, int64_t N, const float *q, const float *U,
                              const float *L, int n, int w, int p, float *out, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    w = min(w, n - 1);
    const int warps = 4;
    size_t smem = (size_t)warps * 4 * n * sizeof(float);
    int blocks = (int)std::min<int64_t>((N + warps - 1) / warps, (int64_t)device_sm_count() * 16);
    if (p == 1) {
        cudaFuncSetAttribute(k_lbi_single<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_lbi_single<1><<<blocks, warps * 32, smem, s>>>(cand, N, q, U, L, n, w, out);
    } else {
        cudaFuncSetAttribute(k_lbi_single<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_lbi_single<2><<<blocks, warps * 32, smem, s>>>(cand, N, q, U, L, n, w, out);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cascade filter over one (query, candidate segment) per CTA:
//   LB_Keogh test  lb[q][c] <= thr                      (Algorithm 3, first test)
//   LB_Improved    lbi = LB_Improved^p <= thr            (second test)
// with thr = b (1 + slack), b the query's current k-th best DTW^p.  Seeds
// (already evaluated) are skipped.  Survivors are collected in shared memory
// and written as one contiguous block of the pair list, whose start and
// length are recorded per (query, segment).
// ---------------------------------------------------------------------------
template <int P>
__global__ void k_lbi_filter(CascadeBufs b) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nw = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.y, sg = blockIdx.x;
    const int n = b.n;
    float *scratch_all = reinterpret_cast<float *>(smraw);
    float *scratch = scratch_all + (size_t)wid * 4 * n;
    int32_t *surv_c = reinterpret_cast<int32_t *>(scratch_all + (size_t)nw * 4 * n);
    float *surv_v = reinterpret_cast<float *>(surv_c + b.seg_len);
    int32_t *seeds = reinterpret_cast<int32_t *>(surv_v + b.seg_len);
    __shared__ int s_count;
    __shared__ unsigned long long s_base;
    __shared__ unsigned long long s_cnt[2];
    if (threadIdx.x == 0) {
        s_count = 0;
        s_cnt[0] = s_cnt[1] = 0;
    }
    for (int t = threadIdx.x; t < b.S; t += blockDim.x) seeds[t] = b.seed_pairs[(int64_t)q * b.S + t].c;
    __syncthreads();

    const float bq = (b.mode == DTW_MODE_NOPRUNE) ? kInf : load_threshold(b.bsf + q);
    const float thr = bq * (1.0f + b.slack);
    const float *y = b.queries + (int64_t)q * n;
    const float *U = b.U + (int64_t)q * n;
    const float *L = b.L + (int64_t)q * n;
    const int c0 = sg * b.seg_len;
    const int c1 = min(b.N, c0 + b.seg_len);
    unsigned long long pk = 0;
    for (int base = c0 + wid * 32; base < c1; base += nw * 32) {
        int c = base + lane;
        bool valid = c < c1;
        float lbv = valid ? b.lb[(int64_t)q * b.N + c] : kInf;
        bool pass = valid && (lbv <= thr);
        if (pass) {
            for (int t = 0; t < b.S; ++t) pass = pass && (seeds[t] != c);
        }
        unsigned m = __ballot_sync(0xffffffffu, pass);
        pk += __popc(m);
        while (m) {
            int src = __ffs(m) - 1;
            m &= m - 1;
            int cc = __shfl_sync(0xffffffffu, c, src);
            float v = __shfl_sync(0xffffffffu, lbv, src);
            if (b.mode == DTW_MODE_IMPROVED) {
                float lbk;
                v = warp_lb_improved<P>(b.db + (int64_t)cc * n, y, U, L, n, b.w, scratch, &lbk);
            }
            if (v <= thr && lane == 0) {
                int slot = atomicAdd(&s_count, 1);
                surv_c[slot] = cc;
                surv_v[slot] = v;
            }
        }
    }
    if (lane == 0) atomicAdd(&s_cnt[0], pk);
    __syncthreads();
    const int cnt = s_count;
    if (threadIdx.x == 0) {
        unsigned long long base = cnt > 0 ? atomicAdd(b.pair_count, (unsigned long long)cnt) : 0ull;
        s_base = base;
        b.seg_start[(int64_t)q * b.nseg + sg] = (int32_t)base;
        b.seg_count[(int64_t)q * b.nseg + sg] = cnt;
        if (b.counters) {
            if (s_cnt[0]) atomicAdd(b.counters + CNT_KEOGH_PASS, s_cnt[0]);
            if (cnt) atomicAdd(b.counters + CNT_LBI_PASS, (unsigned long long)cnt);
        }
    }
    __syncthreads();
    const unsigned long long base = s_base;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        unsigned long long o = base + t;
        b.pairs[o] = Pair{q, surv_c[t]};
        b.pair_lbi[o] = surv_v[t];
        b.pair_res[o] = kInf;
    }
}

cudaError_t launch_lbi_filter(const CascadeBufs &b, cudaStream_t s) {
    if (b.N <= 0 || b.Q <= 0) return cudaSuccess;
    int nw = (int)std::min<int64_t>(8, std::max<int64_t>(1, (160 * 1024) / (16 * (int64_t)b.n)));
    size_t smem = (size_t)nw * 4 * b.n * sizeof(float) + (size_t)b.seg_len * 8 + (size_t)b.S * 4 + 16;
    dim3 grid(b.nseg, b.Q);
    if (b.p == 1) {
        cudaFuncSetAttribute(k_lbi_filter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_lbi_filter<1><<<grid, nw * 32, smem, s>>>(b);
    } else {
        cudaFuncSetAttribute(k_lbi_filter<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_lbi_filter<2><<<grid, nw * 32, smem, s>>>(b);
    }
    return cudaGetLastError();
}

}  // namespace dtwk

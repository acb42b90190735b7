// LB_Keogh (Sec. 7) and LB_Improved (Sec. 8) kernels.
//
//   LB_Keogh_p(x, y)^p    = sum_i d(x_i, [L(y)_i, U(y)_i])^p            (Eq. 1)
//   LB_Improved_p(x, y)^p = LB_Keogh_p(x, y)^p + LB_Keogh_p(y, H(x, y))^p
//
// where H(x, y) clamps x into the envelope of y.  All sums are fp32 in power
// space; the root is taken only where a bound is returned to the caller.
#include <array>
#include <map>
#include <mutex>

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
// pairs of accumulators (4 queries x 4 candidates, even and odd indices),
// summed per chunk and then added to the running total.  Each CTA also writes, per query, the smallest
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
__device__ __forceinline__ void cp_async16_at(unsigned sa, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
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
           unsigned long long *__restrict__ tile_min, int tile0, int ntiles) {
    extern __shared__ __align__(16) unsigned char smraw[];
    TileSmem &sm = *reinterpret_cast<TileSmem *>(smraw);
    // consecutive CTAs share a candidate tile (the database is read once)
    const int q0 = blockIdx.x * TQ;
    const int tile = tile0 + blockIdx.y;
    const int c0 = tile * TC;
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
        // two partial sums per pair (even and odd indices), updated with
        // packed fp32x2 arithmetic: x - U and L - x as fma(., -1, .) (one
        // rounding, as a subtraction), a 3-input max per index, then a packed
        // add (p = 1) or fma (p = 2)
        float2 acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.0f, 0.0f);
        const float *xs = sm.x[buf];
        const float *us = sm.u[buf];
        const float *ls = sm.l[buf];
        const float2 m1 = make_float2(-1.0f, -1.0f);
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
                    float2 s = acc[a][b];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 xx = h ? make_float2(xv[b].z, xv[b].w) : make_float2(xv[b].x, xv[b].y);
                        const float2 uu = h ? make_float2(uv[a].z, uv[a].w) : make_float2(uv[a].x, uv[a].y);
                        const float2 ll = h ? make_float2(lv[a].z, lv[a].w) : make_float2(lv[a].x, lv[a].y);
                        const float2 d1 = __ffma2_rn(uu, m1, xx);  // x - U
                        const float2 d2 = __ffma2_rn(xx, m1, ll);  // L - x
                        const float2 dd = make_float2(max3f(d1.x, d2.x, 0.0f), max3f(d1.y, d2.y, 0.0f));
                        s = (P == 1) ? __fadd2_rn(s, dd) : __ffma2_rn(dd, dd, s);
                    }
                    acc[a][b] = s;
                }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) tot[a][b] += acc[a][b].x + acc[a][b].y;
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
        if (lane == 0 && q < Q && tile_min) tile_min[(int64_t)q * ntiles + tile] = key;
    }
}

int lbk_tiles(int N) { return (N + TC - 1) / TC; }

cudaError_t launch_lbk_tile(const float *db, int N, const float *U, const float *L, int Q, int n,
                            int p, float *lb, unsigned long long *tile_min, cudaStream_t s) {
    if (N <= 0 || Q <= 0) return cudaSuccess;
    bool vec = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(db) & 15) == 0) &&
               ((reinterpret_cast<uintptr_t>(U) & 15) == 0) &&
               ((reinterpret_cast<uintptr_t>(L) & 15) == 0);
    const int ntiles = (N + TC - 1) / TC;
    size_t smem = sizeof(TileSmem);
    auto kern = p == 1 ? (vec ? k_lbk_tile<1, true> : k_lbk_tile<1, false>)
                       : (vec ? k_lbk_tile<2, true> : k_lbk_tile<2, false>);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int t0 = 0; t0 < ntiles; t0 += 65535) {  // grid.y limit
        dim3 grid((Q + TQ - 1) / TQ, std::min(65535, ntiles - t0));
        kern<<<grid, 256, smem, s>>>(db, N, U, L, Q, n, lb, tile_min, t0, ntiles);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// LB_Improved (Sec. 8) of N candidates against one query: the second sum in
// the envelope form derived at the cascade filter below (the candidates'
// envelopes XU, XL and the query's U(L), L(U) computed by the caller); one
// warp per candidate, lane l taking indices l, l + 32, ... (coalesced).
// ---------------------------------------------------------------------------
constexpr int kLbiRegM = 8;  // largest per-lane chunk the filter keeps in registers

struct LbiGeom {
    int m, lg;
};
// M = the power of two >= n/32 (elements per lane), lg = log2(M)
__host__ __device__ inline LbiGeom lbi_geom(int n) {
    LbiGeom g;
    const int need = (n + 31) / 32;
    g.m = 1;
    g.lg = 0;
    while (g.m < need) {
        g.m <<= 1;
        ++g.lg;
    }
    return g;
}

// This lane's elements of a candidate row (MT > 0).
template <int MT>
struct LbiChunk {
    float v[MT > 0 ? MT : 1];
};

template <int P>
__global__ void __launch_bounds__(256)
k_lbi_single(const float *__restrict__ cand, int64_t N, const float *__restrict__ q, const float *__restrict__ U,
             const float *__restrict__ L, const float *__restrict__ XU, const float *__restrict__ XL,
             const float *__restrict__ UL, const float *__restrict__ LU, int n, float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < N; c += warps) {
        const int64_t o = c * n;
        float a1 = 0.0f, a2 = 0.0f;
        for (int i = lane; i < n; i += 32) {
            a1 = acc_dist<P>(a1, __ldg(cand + o + i), __ldg(L + i), __ldg(U + i));
            a2 = acc_dist<P>(a2, __ldg(q + i), fminf(__ldg(XL + o + i), __ldg(LU + i)),
                             fmaxf(__ldg(XU + o + i), __ldg(UL + i)));
        }
        const float v = warp_sum(a1 + a2);
        if (lane == 0) out[c] = root_p(v, P);
    }
}

cudaError_t launch_lbi_single(const float *cand, int64_t N, const float *q, const float *U, const float *L,
                              const float *XU, const float *XL, const float *UL, const float *LU, int n, int p,
                              float *out, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((N + 7) / 8, (int64_t)device_sm_count() * 16);
    if (p == 1) k_lbi_single<1><<<blocks, 256, 0, s>>>(cand, N, q, U, L, XU, XL, UL, LU, n, out);
    else k_lbi_single<2><<<blocks, 256, 0, s>>>(cand, N, q, U, L, XU, XL, UL, LU, n, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cascade filter over one (query, candidate segment) per CTA:
//   pre-filter / LB_Keogh test  lb[q][c] <= thr        (Algorithm 3, first test)
//   LB_Improved                 LB_Improved^p <= thr   (second test)
// with thr = b (1 + slack), b the query's current k-th best DTW^p.  Seeds
// (already evaluated) are skipped.  Survivors are collected in shared memory
// and written as one contiguous block of the pair list, whose start and
// length are recorded per (query, segment, warp).
//
// LB_Improved's second sum, sum_i d(y_i, [L(H)_i, U(H)_i])^p over the
// envelope of the projection H = H(x, y) (Eq. 1), is evaluated as
//
//   sum_i d(y_i, [min(XL_i, LU_i), max(XU_i, UL_i)])^p
//
// with XU, XL the candidate's own envelope (computed once per database row)
// and UL = U(L), LU = L(U) the envelopes of the query's envelope.  The two
// are equal term by term.  H_j = min(max(x_j, L_j), U_j) <= max(x_j, L_j), so
// U(H)_i <= max(XU_i, UL_i): where y_i <= U(H)_i both upper terms are 0.
// Where y_i > U(H)_i, every j in the window of i has i in its own window, so
// U_j >= y_i > U(H)_i >= H_j: no H_j in the window is clipped at U_j, and
// U(H)_i = max_j max(x_j, L_j) = max(XU_i, UL_i).  The lower terms follow by
// symmetry.  Min and max do not round, so each term is the one the
// definition gives; only the order of the fp32 sums differs.  No projection,
// no sliding window and no exchange between lanes remain: each lane adds
// its own indices and one warp reduction closes each sum.
// ---------------------------------------------------------------------------

// Indices of a lane for MT > 0 (no sum here relates different indices, so
// any assignment works; this one makes every copy of a warp contiguous):
// with vector rows, 16-byte pieces lane, lane + 32, ... (index 4 (lane + 32 j)
// + k is element 4 j + k); otherwise indices lane, lane + 32, ...
template <int MT>
__device__ __forceinline__ int env_index(int lane, int t, bool vec) {
    return (vec && MT >= 4) ? 4 * (lane + 32 * (t >> 2)) + (t & 3) : lane + 32 * t;
}

// Query side of the filter for MT > 0: this lane's elements of U, L, y, UL,
// LU (zero beyond the series, where every term is then 0).
template <int MT>
struct EnvQuery {
    float u[MT > 0 ? MT : 1], l[MT > 0 ? MT : 1], y[MT > 0 ? MT : 1], ul[MT > 0 ? MT : 1], lu[MT > 0 ? MT : 1];
};

// UL, LU exist only when the run computes LB_Improved (b.lbi_inline).
template <int MT>
__device__ __forceinline__ void env_load_query(EnvQuery<MT> &Qv, const CascadeBufs &b, int q, bool vec) {
    if constexpr (MT > 0) {
        const int lane = threadIdx.x & 31;
        const int64_t o = (int64_t)q * b.n;
        const bool second = b.lbi_inline != 0;
#pragma unroll
        for (int t = 0; t < MT; ++t) {
            const int i = env_index<MT>(lane, t, vec);
            const bool in = i < b.n;
            Qv.u[t] = in ? b.U[o + i] : 0.0f;
            Qv.l[t] = in ? b.L[o + i] : 0.0f;
            Qv.y[t] = in ? b.queries[o + i] : 0.0f;
            Qv.ul[t] = (in && second) ? b.UL[o + i] : 0.0f;
            Qv.lu[t] = (in && second) ? b.LU[o + i] : 0.0f;
        }
    }
}

// The rows of one candidate this lane reads (MT > 0): its chunk of x (for
// the first sum, when the matrix does not already hold LB_Keogh) and of the
// candidate's envelope XU, XL (for the second).
template <int MT>
struct EnvRows {
    LbiChunk<MT> x, xu, xl;
};

// Rows reach the warp through a ring of kEnvStages stages in shared memory,
// filled by cp.async kEnvStages - 1 pairs ahead of their use.  Each lane
// copies and reads back only its own elements of each row (x, XU, XL), so
// the ring needs no barrier: a lane's wait for its copy group is enough.  A
// stage holds each row in order ([row][32 MT] floats): a warp's copies and
// reads cover contiguous 512-byte (or 128-byte) spans.
constexpr int kEnvStages = 3;
template <int MT>
constexpr int env_ring_floats() {
    return MT > 0 ? kEnvStages * 3 * 32 * MT : 0;
}

// Starts the copies of candidate c's rows into stage st.  XU, XL exist only
// when the run computes LB_Improved (b.lbi_inline); x only when the matrix
// does not already hold LB_Keogh (need_x).  Elements past the series are
// zero-filled (their terms are then 0), their source clamped to the row start.
//
// FAST: rows of exactly 32 MT elements with 16-byte pieces, x and the
// envelope rows all needed (the common case, specialised at compile time:
// no predicates and no clamped sources).
template <int MT, bool FAST>
__device__ __forceinline__ void env_issue(float *ring, int st, const CascadeBufs &b, int c, bool vec, bool need_x) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)c * b.n;
    float *stage = ring + st * 3 * 32 * MT;
    if constexpr (FAST) {
        static_assert(MT >= 4, "16-byte pieces");
        const unsigned sa = (unsigned)__cvta_generic_to_shared(stage) + 16u * lane;
        const float *s0 = b.db + row + 4 * lane, *s1 = b.XU + row + 4 * lane, *s2 = b.XL + row + 4 * lane;
#pragma unroll
        for (int j = 0; j < MT / 4; ++j) {
            cp_async16_at(sa + 512u * j, s0 + 128 * j);
            cp_async16_at(sa + 128u * MT + 512u * j, s1 + 128 * j);
            cp_async16_at(sa + 256u * MT + 512u * j, s2 + 128 * j);
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        if (r == 0 && !need_x) continue;
        if (r > 0 && !b.lbi_inline) continue;
        const float *src = (r == 0 ? b.db : (r == 1 ? b.XU : b.XL)) + row;
        float *dst = stage + r * 32 * MT;
        if (vec && MT >= 4) {
#pragma unroll
            for (int j = 0; j < MT / 4; ++j) {
                const int i = 4 * (lane + 32 * j);  // n % 4 == 0: a piece is wholly in or out
                const bool in = i < b.n;
                cp_async16(dst + i, in ? src + i : src, in);
            }
        } else {
#pragma unroll
            for (int t = 0; t < MT; ++t) {
                const int i = lane + 32 * t;
                const bool in = i < b.n;
                cp_async4(dst + i, in ? src + i : src, in);
            }
        }
    }
}

// This lane's chunks of stage st, after its copies completed.
template <int MT>
__device__ __forceinline__ void env_read(EnvRows<MT> &rw, const float *ring, int st, bool vec, bool need_x,
                                         bool need_env) {
    const int lane = threadIdx.x & 31;
    const float *stage = ring + st * 3 * 32 * MT;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        if (r == 0 && !need_x) continue;
        if (r > 0 && !need_env) continue;
        float *v = r == 0 ? rw.x.v : (r == 1 ? rw.xu.v : rw.xl.v);
        const float *src = stage + r * 32 * MT;
        if (vec && MT >= 4) {
#pragma unroll
            for (int j = 0; j < MT / 4; ++j) {
                const float4 f = *reinterpret_cast<const float4 *>(src + 4 * (lane + 32 * j));
                v[4 * j] = f.x;
                v[4 * j + 1] = f.y;
                v[4 * j + 2] = f.z;
                v[4 * j + 3] = f.w;
            }
        } else {
#pragma unroll
            for (int t = 0; t < MT; ++t) v[t] = src[lane + 32 * t];
        }
    }
}


// LB_Improved^p of the pair (q, c), or LB_Keogh^p alone when that exceeds thr
// or !do_lbi.  known >= 0: LB_Keogh^p already computed (the first sum is not
// formed again).  *lbk gets LB_Keogh^p.  MT > 0: r holds this lane's chunks;
// MT == 0: lane l takes the 16-byte pieces l, l + 32, ... (vec: n % 4 == 0
// and aligned rows) or the indices l, l + 32, ... (coalesced loads).
template <int P, int MT>
__device__ __forceinline__ float warp_lbi_env(const CascadeBufs &b, int q, int c, const EnvQuery<MT> &Qv,
                                              const EnvRows<MT> &r, float known, float thr, bool do_lbi,
                                              float *lbk, bool vec) {
    const int lane = threadIdx.x & 31;
    const int n = b.n;
    if constexpr (MT > 0) {
        if (known < 0.0f && do_lbi) {
            // Registers hold both rows' chunks: form both sums, then reduce
            // them together, so that their shuffle chains overlap (one
            // reduction's latency per pair instead of two in a row).  The
            // second sum of a pair that fails LB_Keogh is formed for nothing
            // (a few percent of the pairs).
            float a1 = 0.0f, a2 = 0.0f;
#pragma unroll
            for (int t = 0; t < MT; ++t) {
                a1 = acc_dist<P>(a1, r.x.v[t], Qv.l[t], Qv.u[t]);
                a2 = acc_dist<P>(a2, Qv.y[t], fminf(r.xl.v[t], Qv.lu[t]), fmaxf(r.xu.v[t], Qv.ul[t]));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a1 += __shfl_xor_sync(0xffffffffu, a1, o);
                a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            }
            *lbk = a1;
            return a1 > thr ? a1 : a1 + a2;
        }
    } else {
        if (known < 0.0f && do_lbi && vec) {
            // Long rows, streamed: both sums in one pass over 16-byte pieces,
            // so that the loads of the two sums are in flight together, and
            // one combined reduction.
            const int64_t oc = (int64_t)c * n, oq = (int64_t)q * n;
            const float *x = b.db + oc, *xu = b.XU + oc, *xl = b.XL + oc;
            const float *U = b.U + oq, *L = b.L + oq, *y = b.queries + oq, *ul = b.UL + oq, *lu = b.LU + oq;
            float a1 = 0.0f, a2 = 0.0f;
            if (b.lb_abandon) {
                // Early abandoning inside the sums (the remark on abandoning
                // the bound sums in the experiments of Sec. 10): every
                // kLbAbandonSpan indices the partial sums, which only grow,
                // are compared with thr.  Above it, LB_Keogh decides at once;
                // if only LB_Keogh + the second sum is, the pair fails
                // LB_Improved whatever the rest, and only LB_Keogh is
                // completed (three of the eight rows) to tell which bound
                // discarded it.
                int base = 0;
                bool lbi_out = false;
                for (; base < n; base += 128) {
                    const int i = base + 4 * lane;
                    if (i < n) {
                        a1 = acc_dist4<P>(a1, ldg4(x + i), ldg4(L + i), ldg4(U + i));
                        a2 = acc_dist4<P>(a2, ldg4(y + i), min4(ldg4(xl + i), ldg4(lu + i)),
                                          max4(ldg4(xu + i), ldg4(ul + i)));
                    }
                    if ((base + 128) % kLbAbandonSpan == 0 && base + 128 < n) {
                        float s1 = a1, s12 = a1 + a2;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                            s12 += __shfl_xor_sync(0xffffffffu, s12, o);
                        }
                        if (s1 > thr) {
                            *lbk = s1;
                            return s1;
                        }
                        if (s12 > thr) {
                            lbi_out = true;
                            base += 128;
                            break;
                        }
                    }
                }
                if (lbi_out) {
                    for (; base < n; base += 128) {
                        const int i = base + 4 * lane;
                        if (i < n) a1 = acc_dist4<P>(a1, ldg4(x + i), ldg4(L + i), ldg4(U + i));
                    }
                    const float s1 = warp_sum(a1);
                    *lbk = s1;
                    return s1 > thr ? s1 : kInf;  // LB_Improved > thr either way
                }
            } else {
#pragma unroll 2
                for (int i = 4 * lane; i < n; i += 128) {
                    a1 = acc_dist4<P>(a1, ldg4(x + i), ldg4(L + i), ldg4(U + i));
                    a2 = acc_dist4<P>(a2, ldg4(y + i), min4(ldg4(xl + i), ldg4(lu + i)),
                                      max4(ldg4(xu + i), ldg4(ul + i)));
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a1 += __shfl_xor_sync(0xffffffffu, a1, o);
                a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            }
            *lbk = a1;
            return a1 > thr ? a1 : a1 + a2;
        }
    }
    float first = known;
    if (known < 0.0f) {
        float acc = 0.0f;
        if constexpr (MT > 0) {
#pragma unroll
            for (int t = 0; t < MT; ++t) acc = acc_dist<P>(acc, r.x.v[t], Qv.l[t], Qv.u[t]);
        } else {
            const float *x = b.db + (int64_t)c * n;
            const float *U = b.U + (int64_t)q * n, *L = b.L + (int64_t)q * n;
            if (vec) {
#pragma unroll 2
                for (int i = 4 * lane; i < n; i += 128) acc = acc_dist4<P>(acc, ldg4(x + i), ldg4(L + i), ldg4(U + i));
            } else {
#pragma unroll 4
                for (int i = lane; i < n; i += 32) acc = acc_dist<P>(acc, __ldg(x + i), __ldg(L + i), __ldg(U + i));
            }
        }
        first = warp_sum(acc);
    }
    *lbk = first;
    if (!do_lbi || first > thr) return first;
    float acc = 0.0f;
    if constexpr (MT > 0) {
#pragma unroll
        for (int t = 0; t < MT; ++t)
            acc = acc_dist<P>(acc, Qv.y[t], fminf(r.xl.v[t], Qv.lu[t]), fmaxf(r.xu.v[t], Qv.ul[t]));
    } else {
        const int64_t oc = (int64_t)c * n, oq = (int64_t)q * n;
        const float *xu = b.XU + oc, *xl = b.XL + oc;
        const float *y = b.queries + oq, *ul = b.UL + oq, *lu = b.LU + oq;
        if (vec) {
#pragma unroll 2
            for (int i = 4 * lane; i < n; i += 128)
                acc = acc_dist4<P>(acc, ldg4(y + i), min4(ldg4(xl + i), ldg4(lu + i)), max4(ldg4(xu + i), ldg4(ul + i)));
        } else {
#pragma unroll 4
            for (int i = lane; i < n; i += 32)
                acc = acc_dist<P>(acc, __ldg(y + i), fminf(__ldg(xl + i), __ldg(lu + i)),
                                  fmaxf(__ldg(xu + i), __ldg(ul + i)));
        }
    }
    // one reduction of the full value keeps the sum's rounding independent
    // of where the first sum came from
    return warp_sum(acc + (lane == 0 ? first : 0.0f));
}

// Phase 1 of a filter segment [c0, c1) for the calling warp: the stored
// bounds of its share of the segment (candidates c0 + wid * 32 + lane, then
// in strides of the CTA's warps) are tested against thr_m, and the
// candidates that pass are compacted, in order, into the warp's buffers
// (seeds hold NaN in the matrix and never pass).  Eight loads per lane are
// issued before any is tested, so that the scan waits on memory once per
// eight rows of 32.  The matrix is read once: its loads are marked
// evict-first, so that the segment's rows, which every query's CTA reads,
// stay in L2.  Returns the number of candidates kept.
__device__ __forceinline__ int scan_segment(const float *__restrict__ lbrow, int c0, int c1, int wid, int stride,
                                            float thr_m, int32_t *surv_c, float *surv_v) {
    const int lane = threadIdx.x & 31;
    int cnt1 = 0;
    for (int base0 = c0 + wid * 32; base0 < c1; base0 += 8 * stride) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = base0 + u * stride + lane;
            v[u] = c < c1 ? __ldcs(lbrow + c) : kInf;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = base0 + u * stride + lane;
            const bool pass = c < c1 && v[u] <= thr_m;
            const unsigned m = __ballot_sync(0xffffffffu, pass);
            if (pass) {
                const int slot = cnt1 + __popc(m & ((1u << lane) - 1));
                surv_c[slot] = c;
                surv_v[slot] = v[u];
            }
            cnt1 += __popc(m);
        }
    }
    __syncwarp();
    return cnt1;
}

// Writes the warp's cnt survivors of segment sg (candidates surv_c, bounds
// surv_v) as one contiguous block of the pair list and records its start and
// length as sub-segment (q, sg, wid); adds the stage counters (cnt1
// candidates passed the stored bound, kp of them LB_Keogh when the matrix
// held the piecewise-sum bound).
__device__ __forceinline__ void emit_survivors(const CascadeBufs &b, int q, int sg, int nsegs, int nw, int wid, int cnt,
                                               int cnt1, unsigned long long kp, const int32_t *surv_c,
                                               const float *surv_v) {
    const int lane = threadIdx.x & 31;
    const unsigned long long pk = (unsigned long long)cnt1;
    unsigned long long base = 0;
    if (lane == 0 && cnt > 0) base = atomicAdd(b.pair_count, (unsigned long long)cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    const int64_t sub = ((int64_t)q * nsegs + sg) * nw + wid;
    if (lane == 0) {
        b.seg_start[sub] = (int32_t)base;
        b.seg_count[sub] = cnt;
        if (cnt) atomicAdd(b.qcount + q, cnt);
        if (b.counters) {
            if (b.summary) {
                if (pk) atomicAdd(b.counters + CNT_SUMMARY_PASS, pk);
                if (kp) atomicAdd(b.counters + CNT_KEOGH_PASS, kp);
            } else if (pk) {
                atomicAdd(b.counters + CNT_KEOGH_PASS, pk);
            }
            if (cnt && b.mode != DTW_MODE_IMPROVED) atomicAdd(b.counters + CNT_LBI_PASS, (unsigned long long)cnt);
            if (cnt && b.lbi_inline) atomicAdd(b.counters + CNT_LBI_PASS, (unsigned long long)cnt);
        }
    }
    __syncwarp();
    for (int t = lane; t < cnt; t += 32) {
        const unsigned long long o = base + t;
        b.pairs_u[o] = Pair{q, surv_c[t]};
        b.lbi_u[o] = surv_v[t];
    }
}

template <int P, int MT, bool FAST>
__global__ void __launch_bounds__(256, 2) k_lbi_filter(CascadeBufs b, bool vec_arg) {
    // FAST (see env_issue): 16-byte rows of exactly 32 MT elements, the
    // pre-filter matrix and LB_Improved on
    const bool vec = FAST ? true : vec_arg;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nw = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // CTAs in flight share a candidate segment (consecutive CTAs are queries),
    // so the segment's rows stay in L2 for all the queries that test them
    const int q = blockIdx.x;
    const int per_warp_cap = b.seg_len / nw + 32;  // candidates one warp scans, rounded up
    float *ring = reinterpret_cast<float *>(smraw) + (size_t)wid * env_ring_floats<MT>();
    int32_t *surv_c = reinterpret_cast<int32_t *>(smraw) + (size_t)nw * env_ring_floats<MT>() +
                      (size_t)wid * 2 * per_warp_cap;
    float *surv_v = reinterpret_cast<float *>(surv_c + per_warp_cap);
    EnvQuery<MT> Qv;
    if (b.lbi_inline || b.summary) env_load_query<MT>(Qv, b, q, vec);

    // From here on each warp works alone: for each of the CTA's segments it
    // scans its share of the segment, keeps its survivors in its own shared
    // buffer and writes them as one contiguous block of the pair list
    // (sub-segment (q, sg, wid)).
    const float bq = (b.mode == DTW_MODE_NOPRUNE) ? kInf : load_threshold(b.bsf + q);
    const float thr = bq * (1.0f + b.slack);
    // the matrix holds LB_Keogh^p, or the piecewise-sum bound in the units of
    // sum_j D_j^p (for p = 2 the bound is that sum over max_j |C_j|)
    const float thr_m = b.summary ? thr * b.summary_scale : thr;
    const int nsegs = b.nseg / nw;
    const bool lbk_done = FAST ? false : !b.summary;  // the survivors carry LB_Keogh^p
    const bool lbi_on = FAST ? true : b.lbi_inline != 0;
    const float *lbrow = b.lb + (int64_t)q * b.N;
    const int stride = nw * 32;
    for (int sj = 0; sj < b.seg_per_cta; ++sj) {
    const int sg = blockIdx.y * b.seg_per_cta + sj;
    if (sg >= nsegs) break;
    const int c0 = sg * b.seg_len;
    const int c1 = min(b.N, c0 + b.seg_len);
    const int cnt1 = scan_segment(lbrow, c0, c1, wid, stride, thr_m, surv_c, surv_v);
    unsigned long long kp = 0;  // LB_Keogh survivors (summary mode)
    // phase 2: LB_Keogh (when the matrix held the pre-filter bound) and
    // LB_Improved of each survivor, warp per pair, the rows of the next
    // kEnvStages - 1 candidates in flight (MT > 0) while the current one is
    // processed; survivors are kept in place (write index <= read index)
    int cnt = 0;
    if (lbi_on || !lbk_done) {
        const bool need_x = !lbk_done;
        if constexpr (MT > 0) {
#pragma unroll
            for (int e = 0; e < kEnvStages - 1; ++e) {
                if (e < cnt1) env_issue<MT, FAST>(ring, e, b, surv_c[e], vec, need_x);
                cp_async_commit();
            }
        }
        for (int e = 0; e < cnt1; ++e) {
            const int cc = surv_c[e];
            const float known = lbk_done ? surv_v[e] : -1.0f;
            EnvRows<MT> cur;
            if constexpr (MT > 0) {
                // the stage refilled here was read (and used) by pair e - 1
                const int ahead = e + kEnvStages - 1;
                if (ahead < cnt1) env_issue<MT, FAST>(ring, ahead % kEnvStages, b, surv_c[ahead], vec, need_x);
                cp_async_commit();
                cp_async_wait<kEnvStages - 1>();
                env_read<MT>(cur, ring, e % kEnvStages, vec, need_x, lbi_on);
            }
            float lbk;
            const float v = warp_lbi_env<P, MT>(b, q, cc, Qv, cur, known, thr, lbi_on, &lbk, vec);
            if (!lbk_done) kp += (lbk <= thr) ? 1 : 0;
            if (v <= thr) {
                if (lane == 0) {
                    surv_c[cnt] = cc;
                    surv_v[cnt] = v;
                    // the survivor's matrix entry becomes its LB_Keogh^p (the
                    // DTW stage's cumulative bound starts from it)
                    if (!lbk_done) b.lb[(int64_t)q * b.N + cc] = lbk;
                }
                ++cnt;
            }
            __syncwarp();
        }
        if constexpr (MT > 0) cp_async_wait<0>();  // only empty groups remain
    } else {
        cnt = cnt1;
    }
    emit_survivors(b, q, sg, nsegs, nw, wid, cnt, cnt1, kp, surv_c, surv_v);
    __syncwarp();  // the survivor buffer is refilled by the next segment
    }  // segments of this CTA
}

// ---------------------------------------------------------------------------
// Query terms and pair sums of the batched filter (k_lbi_batch below), in
// packed fp32x2 arithmetic: lane l holds the query terms of its 16-byte
// pieces l, l + 32, ... of a row of 32 MT elements, two indices per float2.
// The second sum's term is restated as
//   d(y, [min(XL, LU), max(XU, UL)]) = max(min(y - XU, A), min(XL - y, B), 0)
// with the per-query constants A = y - U(L) and B = L(U) - y: rounding is
// monotone, so fl(y - max(XU, UL)) = min(fl(y - XU), fl(y - UL)) and
// fl(min(XL, LU) - y) = min(fl(XL - y), fl(LU - y)), and every term equals
// the one k_lbi_filter forms.
// ---------------------------------------------------------------------------
template <int MT>
struct QueryPacked {
    float2 u[MT / 2], l[MT / 2], y[MT / 2], a[MT / 2], b[MT / 2];
};

template <int MT>
struct RowsPacked {
    float4 x[MT / 4], xu[MT / 4], xl[MT / 4];
};

template <int MT>
__device__ __forceinline__ void query_load_packed(QueryPacked<MT> &Q, const CascadeBufs &b, int q) {
    const int lane = threadIdx.x & 31;
    const int64_t o = (int64_t)q * (32 * MT) + 4 * lane;
#pragma unroll
    for (int j = 0; j < MT / 4; ++j) {
        const float4 u = ldg4(b.U + o + 128 * j), l = ldg4(b.L + o + 128 * j), y = ldg4(b.queries + o + 128 * j);
        const float4 ul = ldg4(b.UL + o + 128 * j), lu = ldg4(b.LU + o + 128 * j);
        Q.u[2 * j] = make_float2(u.x, u.y);
        Q.u[2 * j + 1] = make_float2(u.z, u.w);
        Q.l[2 * j] = make_float2(l.x, l.y);
        Q.l[2 * j + 1] = make_float2(l.z, l.w);
        Q.y[2 * j] = make_float2(y.x, y.y);
        Q.y[2 * j + 1] = make_float2(y.z, y.w);
        Q.a[2 * j] = make_float2(y.x - ul.x, y.y - ul.y);
        Q.a[2 * j + 1] = make_float2(y.z - ul.z, y.w - ul.w);
        Q.b[2 * j] = make_float2(lu.x - y.x, lu.y - y.y);
        Q.b[2 * j + 1] = make_float2(lu.z - y.z, lu.w - y.w);
    }
}

// This lane's parts of LB_Keogh^p (s1) and of the second sum (s2) of one pair.
// Each sum is split over two accumulators (even and odd t) so that the adds
// form two short chains instead of one long one; any order of these
// non-negative terms is covered by the slack of the pruning tests.
template <int P, int MT>
__device__ __forceinline__ void pair_sums(const QueryPacked<MT> &Q, const RowsPacked<MT> &r, float &s1, float &s2) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    float2 a1[2] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
    float2 a2[2] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
#pragma unroll
    for (int j = 0; j < MT / 4; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = 2 * j + h;
            const float2 x = h ? make_float2(r.x[j].z, r.x[j].w) : make_float2(r.x[j].x, r.x[j].y);
            const float2 xu = h ? make_float2(r.xu[j].z, r.xu[j].w) : make_float2(r.xu[j].x, r.xu[j].y);
            const float2 xl = h ? make_float2(r.xl[j].z, r.xl[j].w) : make_float2(r.xl[j].x, r.xl[j].y);
            const float2 d1 = __ffma2_rn(Q.u[t], m1, x);  // x - U
            const float2 d2 = __ffma2_rn(x, m1, Q.l[t]);  // L - x
            const float2 k = make_float2(max3f(d1.x, d2.x, 0.0f), max3f(d1.y, d2.y, 0.0f));
            a1[h] = (P == 1) ? __fadd2_rn(a1[h], k) : __ffma2_rn(k, k, a1[h]);
            const float2 e1 = __ffma2_rn(xu, m1, Q.y[t]);  // y - XU
            const float2 e2 = __ffma2_rn(Q.y[t], m1, xl);  // XL - y
            const float2 g = make_float2(max3f(fminf(e1.x, Q.a[t].x), fminf(e2.x, Q.b[t].x), 0.0f),
                                         max3f(fminf(e1.y, Q.a[t].y), fminf(e2.y, Q.b[t].y), 0.0f));
            a2[h] = (P == 1) ? __fadd2_rn(a2[h], g) : __ffma2_rn(g, g, a2[h]);
        }
    const float2 b1 = __fadd2_rn(a1[0], a1[1]), b2 = __fadd2_rn(a2[0], a2[1]);
    s1 = b1.x + b1.y;
    s2 = b2.x + b2.y;
}

// ---------------------------------------------------------------------------
// Filter with batched reductions: the compiled fast case of k_lbi_filter
// (rows of exactly 32 MT elements, MT = 4 or 8, 16-byte pieces, the
// piecewise-sum pre-filter and LB_Improved on), with the same row ring, the
// same terms (formed by pair_sums above) and the same tests, but the pairs
// of a warp taken eight at a time.  Each lane keeps its partial sums of the eight pairs (LB_Keogh and
// the second sum: 16 values) in registers; one transposed butterfly then
// reduces all 16 over the warp (each exchange step halves the values a lane
// holds), so that lane 2j ends with pair j's LB_Keogh and lane 16 + 2j with
// its second sum.  The eight decisions and the survivors' compaction are
// made by eight lanes at once.  Against one reduction chain and one round of
// single-lane bookkeeping per pair, this removes about half of the
// instructions a pair costs and the serial shuffle latency between pairs.
// ---------------------------------------------------------------------------

template <int P, int MT>
__global__ void __launch_bounds__(256, 2) k_lbi_batch(CascadeBufs b) {
    static_assert(MT == 4 || MT == 8, "rows of 128 or 256 elements");
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nw = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.x;
    const int per_warp_cap = b.seg_len / nw + 32;
    float *ring = reinterpret_cast<float *>(smraw) + (size_t)wid * env_ring_floats<MT>();
    int32_t *surv_c = reinterpret_cast<int32_t *>(smraw) + (size_t)nw * env_ring_floats<MT>() +
                      (size_t)wid * 2 * per_warp_cap;
    float *surv_v = reinterpret_cast<float *>(surv_c + per_warp_cap);
    QueryPacked<MT> Qp;
    query_load_packed<MT>(Qp, b, q);
    const float bq = (b.mode == DTW_MODE_NOPRUNE) ? kInf : load_threshold(b.bsf + q);
    const float thr = bq * (1.0f + b.slack);
    const float thr_m = thr * b.summary_scale;  // the matrix holds the piecewise-sum bound
    const int nsegs = b.nseg / nw;
    float *lbrow = b.lb + (int64_t)q * b.N;
    const int stride = nw * 32;
    for (int sj = 0; sj < b.seg_per_cta; ++sj) {
        const int sg = blockIdx.y * b.seg_per_cta + sj;
        if (sg >= nsegs) break;
        const int c0 = sg * b.seg_len;
        const int c1 = min(b.N, c0 + b.seg_len);
        const int cnt1 = scan_segment(lbrow, c0, c1, wid, stride, thr_m, surv_c, surv_v);
        unsigned long long kp = 0;
        int cnt = 0;
#pragma unroll
        for (int e = 0; e < kEnvStages - 1; ++e) {
            if (e < cnt1) env_issue<MT, true>(ring, e, b, surv_c[e], true, true);
            cp_async_commit();
        }
        int st = 0;  // stage of pair e (e % kEnvStages), kept by increments
        for (int e0 = 0; e0 < cnt1; e0 += kLbiBatch) {
            float v[16];
#pragma unroll
            for (int u = 0; u < kLbiBatch; ++u) {
                const int e = e0 + u;
                float a1 = 0.0f, a2 = 0.0f;
                if (e < cnt1) {
                    // the stage refilled here, (e + 2) % 3, was read (and used) by pair e - 1
                    static_assert(kEnvStages == 3, "stage arithmetic below");
                    const int ahead = e + kEnvStages - 1;
                    const int st_ahead = st == 0 ? 2 : st - 1;
                    if (ahead < cnt1) env_issue<MT, true>(ring, st_ahead, b, surv_c[ahead], true, true);
                    cp_async_commit();
                    cp_async_wait<kEnvStages - 1>();
                    RowsPacked<MT> R;
                    const float *stage = ring + (size_t)st * 3 * 32 * MT;
                    st = st == 2 ? 0 : st + 1;
#pragma unroll
                    for (int jj = 0; jj < MT / 4; ++jj) {
                        R.x[jj] = *reinterpret_cast<const float4 *>(stage + 4 * (lane + 32 * jj));
                        R.xu[jj] = *reinterpret_cast<const float4 *>(stage + 32 * MT + 4 * (lane + 32 * jj));
                        R.xl[jj] = *reinterpret_cast<const float4 *>(stage + 64 * MT + 4 * (lane + 32 * jj));
                    }
                    pair_sums<P, MT>(Qp, R, a1, a2);
                }
                v[u] = a1;
                v[u + 8] = a2;
            }
            // lane 2j: pair j's LB_Keogh^p; lane 16 + 2j: its second sum
            const float s1 = warp_sum16_transposed(v);
            const float s2 = __shfl_down_sync(0xffffffffu, s1, 16);
            const int j = lane >> 1;
            const bool decides = lane < 16 && !(lane & 1) && e0 + j < cnt1;
            const int cc = decides ? surv_c[e0 + j] : 0;
            const float val = s1 > thr ? s1 : s1 + s2;
            const bool pass = decides && val <= thr;
            const unsigned m = __ballot_sync(0xffffffffu, pass);
            kp += __popc(__ballot_sync(0xffffffffu, decides && s1 <= thr));
            __syncwarp();  // every decider has read its candidate before the list is rewritten
            if (pass) {
                const int r = cnt + __popc(m & ((1u << lane) - 1));
                surv_c[r] = cc;  // r <= e0 + j: survivors stay in place or move down
                surv_v[r] = val;
                lbrow[cc] = s1;  // LB_Keogh^p, where the DTW stage's cumulative bound starts
            }
            cnt += __popc(m);
            __syncwarp();
        }
        cp_async_wait<0>();  // only empty groups remain
        emit_survivors(b, q, sg, nsegs, nw, wid, cnt, cnt1, kp, surv_c, surv_v);
        __syncwarp();  // the survivor buffer is refilled by the next segment
    }
}

// chunk length the filter keeps in registers (0: strided loads)
static int lbi_filter_mt(int n) {
    const int m = lbi_geom(n).m;
    return m <= kLbiRegM ? m : 0;
}

static size_t lbi_filter_smem(int n, int S, int seg_len, int nw) {
    (void)S;
    const int mt = lbi_filter_mt(n);
    const int64_t ring = mt > 0 ? (int64_t)kEnvStages * 3 * 32 * mt * 4 : 0;
    return (size_t)(nw * ring + 64 + (int64_t)nw * 8 * (seg_len / nw + 32));
}

// Warps per filter CTA: `want` (1..8) if its shared memory fits, else 8 (the
// CTA's segments and query are then shared by the most warps).
int lbi_filter_warps(int n, int w, int S, int seg_len, int p, int want) {
    (void)w;
    (void)p;
    int nw = (want > 0 && want < 8) ? want : 8;
    while (nw > 1 && lbi_filter_smem(n, S, seg_len, nw) > 227 * 1024) --nw;
    return nw;
}

template <int P, int MT>
static void lbi_filter_go(const CascadeBufs &b, bool vec, cudaStream_t s) {
    const int nw = b.filter_warps > 0 ? b.filter_warps : lbi_filter_warps(b.n, b.w, b.S, b.seg_len, P);
    const size_t smem = lbi_filter_smem(b.n, b.S, b.seg_len, nw);
    const int nsegs = b.nseg / nw;
    const dim3 grid(b.Q, (nsegs + b.seg_per_cta - 1) / b.seg_per_cta);
    const bool fast = MT >= 4 && vec && b.n == 32 * MT && b.summary && b.lbi_inline;
    auto kern = fast ? k_lbi_filter<P, MT, (MT >= 4)> : k_lbi_filter<P, MT, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, nw * 32, smem, s>>>(b, vec);
}

template <int P>
static void lbi_filter_dispatch(const CascadeBufs &b, bool vec, cudaStream_t s) {
    switch (lbi_geom(b.n).m) {
        case 1: lbi_filter_go<P, 1>(b, vec, s); break;
        case 2: lbi_filter_go<P, 2>(b, vec, s); break;
        case 4: lbi_filter_go<P, 4>(b, vec, s); break;
        case 8: lbi_filter_go<P, 8>(b, vec, s); break;
        default: lbi_filter_go<P, 0>(b, vec, s); break;
    }
}

bool lbi_batch_applies(int n, bool summary, bool lbi_inline) { return (n == 128 || n == 256) && summary && lbi_inline; }

template <int P, int MT>
static void lbi_batch_go(const CascadeBufs &b, cudaStream_t s) {
    const int nw = b.filter_warps;
    const size_t smem = lbi_filter_smem(b.n, b.S, b.seg_len, nw);
    const int nsegs = b.nseg / nw;
    const dim3 grid(b.Q, (nsegs + b.seg_per_cta - 1) / b.seg_per_cta);
    auto kern = k_lbi_batch<P, MT>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, nw * 32, smem, s>>>(b);
}

cudaError_t launch_lbi_filter(const CascadeBufs &b, cudaStream_t s) {
    if (b.N <= 0 || b.Q <= 0) return cudaSuccess;
    if (b.lbi_inline && (b.XU == nullptr || b.XL == nullptr || b.UL == nullptr || b.LU == nullptr))
        return cudaErrorInvalidValue;
    // rows start on 16-byte boundaries when n % 4 == 0 and the bases do (the
    // envelope rows and the query envelopes always do)
    const bool vec = (b.n % 4 == 0) && ((reinterpret_cast<uintptr_t>(b.db) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(b.queries) & 15) == 0);
    if (b.filter_path == 2 && vec && lbi_batch_applies(b.n, b.summary != 0, b.lbi_inline != 0)) {
        if (b.n == 256) {
            if (b.p == 1) lbi_batch_go<1, 8>(b, s);
            else lbi_batch_go<2, 8>(b, s);
        } else {
            if (b.p == 1) lbi_batch_go<1, 4>(b, s);
            else lbi_batch_go<2, 4>(b, s);
        }
        return cudaGetLastError();
    }
    if (b.p == 1) lbi_filter_dispatch<1>(b, vec, s);
    else lbi_filter_dispatch<2>(b, vec, s);
    return cudaGetLastError();
}

}  // namespace dtwk

// Warping envelope (Sec. 5): U(y)_i = max_{|k-i|<=w} y_k, L(y)_i = min_{|k-i|<=w} y_k,
// with k clipped to the series.  The paper's Algorithm 1 (Sec. 6) is a
// sequential monotone-deque scan; on the GPU one CTA per series builds a
// sparse table by doubling in shared memory instead:
//   T_0 = y,  T_j[i] = max(T_{j-1}[i], T_{j-1}[min(i + 2^(j-1), n-1)]),
// so T_j[i] is the maximum over [i, min(i + 2^j - 1, n-1)].  A clipped window
// [a, b] of length len has floor(log2(len)) in {kmax-1, kmax}, with
// kmax = floor(log2(min(2w+1, n))), and its maximum is
// max(T_k[a], T_k[b - 2^k + 1]).  Min and max do not round, so the result is
// bit-identical to the definition.
//
// The same kernel optionally writes the four shifted, +INF-padded copies of
// each series that the DTW kernels read their band windows from, and the
// second-order envelopes U(L(y)) and L(U(y)) that LB_Improved's second sum
// takes for the query (Sec. 8; see the filter in lb.cu).
#include "common.cuh"

namespace dtwk {

constexpr int kEnvThreads = 256;

__device__ __forceinline__ int floor_log2(int v) { return 31 - __clz(v); }

// Max table over amax[0..n) and min table over amin[0..n) (both in shared
// memory, ax/an on entry), then U_i = max over the clipped window of i from
// the first and L_i = min from the second.  Ends with a barrier.
__device__ void envelope_windows(float *ax, float *an, float *bx, float *bn, int n, int w, float *__restrict__ Ur,
                                 float *__restrict__ Lr) {
    __syncthreads();
    const int len_max = min(2 * w + 1, n);
    const int kmax = floor_log2(len_max);
    for (int j = 1; j <= kmax; ++j) {
        const int h = 1 << (j - 1);
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            int i2 = min(i + h, n - 1);
            bx[i] = fmaxf(ax[i], ax[i2]);
            bn[i] = fminf(an[i], an[i2]);
        }
        __syncthreads();
        float *t;
        t = ax; ax = bx; bx = t;
        t = an; an = bn; bn = t;
    }
    // now ax/an = T_kmax and bx/bn = T_(kmax-1) (unused when kmax == 0)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int a = max(0, i - w), b = min(n - 1, i + w);
        int k = floor_log2(b - a + 1);
        const float *tx = (k == kmax) ? ax : bx;
        const float *tn = (k == kmax) ? an : bn;
        int b2 = b - (1 << k) + 1;
        Ur[i] = fmaxf(tx[a], tx[b2]);
        Lr[i] = fminf(tn[a], tn[b2]);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kEnvThreads)
k_envelope(const float *__restrict__ y, int n, int w, float *__restrict__ U, float *__restrict__ L,
           float *__restrict__ UL, float *__restrict__ LU, float *__restrict__ copies, int padl, int ylen) {
    extern __shared__ float sm[];
    float *ax = sm, *an = sm + n, *bx = sm + 2 * n, *bn = sm + 3 * n;
    const int64_t row = blockIdx.x;
    const float *yr = y + row * (int64_t)n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        float v = yr[i];
        ax[i] = v;
        an[i] = v;
    }
    if (copies != nullptr) {
        float *cr = copies + row * 4 * (int64_t)ylen;
        for (int t = threadIdx.x; t < 4 * ylen; t += blockDim.x) {
            int r = t / ylen, tt = t - r * ylen;
            int j = tt + r - padl;
            cr[t] = (j >= 0 && j < n) ? yr[j] : kInf;
        }
    }
    float *Ur = U + row * (int64_t)n;
    float *Lr = L + row * (int64_t)n;
    envelope_windows(ax, an, bx, bn, n, w, Ur, Lr);
    if (UL == nullptr) return;
    // second order: the max table over L(y) and the min table over U(y)
    // (written above by this block, visible after the barrier)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        ax[i] = Lr[i];
        an[i] = Ur[i];
    }
    envelope_windows(ax, an, bx, bn, n, w, UL + row * (int64_t)n, LU + row * (int64_t)n);
}

// Many short series (the database rows, once per call): one warp per series,
// the same doubling table in the warp's own shared memory, so that a level
// costs a warp barrier instead of a block barrier.
constexpr int kEnvWarpMaxN = 1024;
constexpr int kEnvWarps = 8;

__global__ void __launch_bounds__(kEnvWarps * 32)
k_envelope_rows(const float *__restrict__ y, int64_t count, int n, int w, float *__restrict__ U,
                float *__restrict__ L) {
    extern __shared__ float sm[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * kEnvWarps + wid;
    if (row >= count) return;
    float *ax = sm + (size_t)wid * 4 * n, *an = ax + n, *bx = ax + 2 * n, *bn = ax + 3 * n;
    const float *yr = y + row * (int64_t)n;
    for (int i = lane; i < n; i += 32) {
        const float v = yr[i];
        ax[i] = v;
        an[i] = v;
    }
    __syncwarp();
    const int kmax = floor_log2(min(2 * w + 1, n));
    for (int j = 1; j <= kmax; ++j) {
        const int h = 1 << (j - 1);
        for (int i = lane; i < n; i += 32) {
            const int i2 = min(i + h, n - 1);
            bx[i] = fmaxf(ax[i], ax[i2]);
            bn[i] = fminf(an[i], an[i2]);
        }
        __syncwarp();
        float *t;
        t = ax; ax = bx; bx = t;
        t = an; an = bn; bn = t;
    }
    float *Ur = U + row * (int64_t)n, *Lr = L + row * (int64_t)n;
    for (int i = lane; i < n; i += 32) {
        const int a = max(0, i - w), b = min(n - 1, i + w);
        const int k = floor_log2(b - a + 1);
        const float *tx = (k == kmax) ? ax : bx;
        const float *tn = (k == kmax) ? an : bn;
        const int b2 = b - (1 << k) + 1;
        Ur[i] = fmaxf(tx[a], tx[b2]);
        Lr[i] = fminf(tn[a], tn[b2]);
    }
}

// Many rows with windows at least as long as a lane's run of outputs: one
// warp per row, the row in shared memory (one padding word per 32 so that
// the lanes' strided reads fall in distinct banks).  Lane l takes the MT
// consecutive outputs [s, e), s = l MT.  Every one of their windows holds the
// common span [max(0, e-1-w), min(n-1, s+w)] (2w + 1 >= MT); the output i
// adds the elements of its own window left of the span (one more per step
// from e-1 down to s) and right of it (one more per step from s up), so a
// lane reads 2w + MT elements for MT outputs instead of a table per level.
// Min and max do not round: the values are the definition's.
__device__ __forceinline__ int env_pad(int i) { return i + (i >> 5); }

template <int MT>
__global__ void __launch_bounds__(kEnvWarps * 32)
k_envelope_runs(const float *__restrict__ y, int64_t count, int n, int w, float *__restrict__ U,
                float *__restrict__ L, bool vec) {
    extern __shared__ float sm[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * kEnvWarps + wid;
    if (row >= count) return;
    float *xs = sm + (size_t)wid * (n + (n >> 5) + 1);
    const float *yr = y + row * (int64_t)n;
    if (vec) {
        for (int i = 4 * lane; i < n; i += 128) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(yr + i));
            xs[env_pad(i)] = v.x;
            xs[env_pad(i + 1)] = v.y;
            xs[env_pad(i + 2)] = v.z;
            xs[env_pad(i + 3)] = v.w;
        }
    } else {
        for (int i = lane; i < n; i += 32) xs[env_pad(i)] = __ldg(yr + i);
    }
    __syncwarp();
    const int s0 = lane * MT;
    if (s0 < n) {
        const int e = min(s0 + MT, n);
        const int lo = max(0, e - 1 - w), hi = min(n - 1, s0 + w);
        float cx = -kInf, cn = kInf;
        int k = lo;
        for (; k + 1 <= hi; k += 2) {
            const float a = xs[env_pad(k)], b = xs[env_pad(k + 1)];
            cx = max3f(cx, a, b);
            cn = min3f(cn, a, b);
        }
        if (k <= hi) {
            const float a = xs[env_pad(k)];
            cx = fmaxf(cx, a);
            cn = fminf(cn, a);
        }
        float ux[MT], ln[MT];
        // right of the span: x[s0 + w + 1 .. i + w]
        float rx = -kInf, rn = kInf;
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            const int j = s0 + m + w;
            if (m > 0 && j <= n - 1) {
                const float v = xs[env_pad(j)];
                rx = fmaxf(rx, v);
                rn = fminf(rn, v);
            }
            ux[m] = fmaxf(cx, rx);
            ln[m] = fminf(cn, rn);
        }
        // left of the span: x[i - w .. e - 2 - w]
        float lx = -kInf, lnn = kInf;
#pragma unroll
        for (int m = MT - 1; m >= 0; --m) {
            const int i = s0 + m;
            if (i < e - 1 && i - w >= 0) {
                const float v = xs[env_pad(i - w)];
                lx = fmaxf(lx, v);
                lnn = fminf(lnn, v);
            }
            ux[m] = fmaxf(ux[m], lx);
            ln[m] = fminf(ln[m], lnn);
        }
        float *Ur = U + row * (int64_t)n + s0, *Lr = L + row * (int64_t)n + s0;
        if (vec && e - s0 == MT && MT >= 4) {
#pragma unroll
            for (int m = 0; m < MT; m += 4) {
                *reinterpret_cast<float4 *>(Ur + m) = make_float4(ux[m], ux[m + 1], ux[m + 2], ux[m + 3]);
                *reinterpret_cast<float4 *>(Lr + m) = make_float4(ln[m], ln[m + 1], ln[m + 2], ln[m + 3]);
            }
        } else {
#pragma unroll
            for (int m = 0; m < MT; ++m)
                if (s0 + m < e) {
                    Ur[m] = ux[m];
                    Lr[m] = ln[m];
                }
        }
    }
}

template <int MT>
static cudaError_t envelope_runs_go(const float *y, int64_t count, int n, int w, float *U, float *L, bool vec,
                                    cudaStream_t s) {
    const size_t smem = (size_t)kEnvWarps * (n + (n >> 5) + 1) * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_envelope_runs<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kEnvWarps * (kEnvWarpMaxN + kEnvWarpMaxN / 32 + 1) * (int)sizeof(float));
        attr = true;
    }
    const int64_t blocks = (count + kEnvWarps - 1) / kEnvWarps;
    k_envelope_runs<MT><<<(unsigned)blocks, kEnvWarps * 32, smem, s>>>(y, count, n, w, U, L, vec);
    return cudaGetLastError();
}

cudaError_t launch_envelope(const float *y, int64_t count, int n, int w, float *U, float *L,
                            QueryCopies qc, int copies_padl, cudaStream_t s, float *UL, float *LU) {
    if (count <= 0) return cudaSuccess;
    if ((UL == nullptr) != (LU == nullptr)) return cudaErrorInvalidValue;
    w = min(w, n - 1);
    if (qc.data == nullptr && UL == nullptr && n <= kEnvWarpMaxN && count >= 4096) {
        // a lane's run of MT outputs (the power of two >= n / 32)
        int mt = 1;
        while (32 * mt < n) mt *= 2;
        if (2 * w + 1 >= mt) {
            const bool vec = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(y) & 15) == 0) &&
                             ((reinterpret_cast<uintptr_t>(U) & 15) == 0) &&
                             ((reinterpret_cast<uintptr_t>(L) & 15) == 0);
            switch (mt) {
                case 1: return envelope_runs_go<1>(y, count, n, w, U, L, vec, s);
                case 2: return envelope_runs_go<2>(y, count, n, w, U, L, vec, s);
                case 4: return envelope_runs_go<4>(y, count, n, w, U, L, vec, s);
                case 8: return envelope_runs_go<8>(y, count, n, w, U, L, vec, s);
                case 16: return envelope_runs_go<16>(y, count, n, w, U, L, vec, s);
                case 32: return envelope_runs_go<32>(y, count, n, w, U, L, vec, s);
                default: break;
            }
        }
        const size_t smem = (size_t)kEnvWarps * 4 * n * sizeof(float);
        static bool rows_attr = false;
        if (!rows_attr) {
            cudaFuncSetAttribute(k_envelope_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kEnvWarps * 4 * kEnvWarpMaxN * (int)sizeof(float));
            rows_attr = true;
        }
        const int64_t blocks = (count + kEnvWarps - 1) / kEnvWarps;
        k_envelope_rows<<<(unsigned)blocks, kEnvWarps * 32, smem, s>>>(y, count, n, w, U, L);
        return cudaGetLastError();
    }
    size_t smem = 4 * (size_t)n * sizeof(float);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_envelope, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             4 * DTW_MAX_N * (int)sizeof(float));
        attr_set = true;
    }
    k_envelope<<<(unsigned)count, kEnvThreads, smem, s>>>(y, n, w, U, L, UL, LU, qc.data, copies_padl,
                                                          qc.ylen);
    return cudaGetLastError();
}

}  // namespace dtwk

// Piecewise-sum bound of Sec. 9.  P_d(x)_j = sum_{i in C_j} x_i over the cover
// C_j = [j s, (j+1) s) for j < d - 1 and C_{d-1} = [(d-1) s, n), s = floor(n/d).
// With D_j = d(P_d(x)_j, [P_d(L)_j, P_d(U)_j]), sum_j D_j <= LB_Keogh_1 (the
// paper's chain of inequalities) and sum_j D_j^2 / max_j |C_j| <= LB_Keogh_2^2
// (Cauchy-Schwarz on each part).  In the cascade the bound of every pair is
// the LB_Keogh tile kernel run on the d part sums (n -> d), which costs 1/s of
// LB_Keogh; LB_Keogh itself is then computed only for its survivors.
#include "common.cuh"

namespace dtwk {

// One thread per (candidate, part); a warp covers consecutive parts of a row.
__global__ void k_summarize(const float *__restrict__ db, int64_t N, int n, int d, int s,
                            float *__restrict__ PX, unsigned *__restrict__ xmax_bits) {
    const int64_t total = N * (int64_t)d;
    float amax = 0.0f;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = o / d;
        const int j = (int)(o - c * d);
        const int lo = j * s, hi = (j == d - 1) ? n : lo + s;
        const float *x = db + c * n;
        float sum = 0.0f;
        for (int i = lo; i < hi; ++i) {
            const float v = __ldg(x + i);
            sum += v;
            amax = fmaxf(amax, fabsf(v));
        }
        PX[o] = sum;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0 && xmax_bits) atomicMax(xmax_bits, __float_as_uint(amax));
}

cudaError_t launch_summarize(const float *db, int64_t N, int n, int d, float *PX, unsigned *xmax_bits,
                             cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const PartGeom g = part_geom(n, d);
    const int64_t total = N * (int64_t)d;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)device_sm_count() * 16);
    k_summarize<<<blocks, 256, 0, s>>>(db, N, n, d, g.s, PX, xmax_bits);
    return cudaGetLastError();
}

// One warp per query: part sums of U and L.  With widen, each part's interval
// is enlarged by delta = 2 smax^2 u (max|x| + max(|U|,|L|)), at least twice
// the worst-case absolute rounding of the difference of two fp32 sums of
// smax terms, so that the fp32 D_j never exceeds the exact one.
__global__ void k_query_summary(const float *__restrict__ U, const float *__restrict__ L, int64_t Q, int n,
                                int d, int s, int smax, const unsigned *__restrict__ xmax_bits,
                                float *__restrict__ PU, float *__restrict__ PL, int widen) {
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (q >= Q) return;
    const float *u = U + q * n, *l = L + q * n;
    float delta = 0.0f;
    if (widen) {
        float m = 0.0f;
        for (int i = lane; i < n; i += 32) m = fmaxf(m, fmaxf(fabsf(u[i]), fabsf(l[i])));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const float xm = xmax_bits ? __uint_as_float(*xmax_bits) : 0.0f;
        delta = 2.0f * (float)smax * (float)smax * 5.9604645e-8f * (xm + m);
    }
    for (int j = lane; j < d; j += 32) {
        const int lo = j * s, hi = (j == d - 1) ? n : lo + s;
        float su = 0.0f, sl = 0.0f;
        for (int i = lo; i < hi; ++i) {
            su += u[i];
            sl += l[i];
        }
        PU[q * d + j] = su + delta;
        PL[q * d + j] = sl - delta;
    }
}

cudaError_t launch_query_summary(const float *U, const float *L, int64_t Q, int n, int d,
                                 const unsigned *xmax_bits, float *PU, float *PL, int widen, cudaStream_t s) {
    if (Q <= 0) return cudaSuccess;
    const PartGeom g = part_geom(n, d);
    const int per = 4;
    k_query_summary<<<(unsigned)((Q + per - 1) / per), 32 * per, 0, s>>>(U, L, Q, n, d, g.s, g.smax, xmax_bits,
                                                                          PU, PL, widen);
    return cudaGetLastError();
}

// Standalone bound of every candidate against one envelope (no widening):
// scratch holds PX [N][d], PU [d], PL [d].
template <int P>
__global__ void k_lbp_single(const float *__restrict__ PX, int64_t N, const float *__restrict__ PU,
                             const float *__restrict__ PL, int d, int smax, float *__restrict__ out) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int j = 0; j < d; ++j) acc = acc_dist<P>(acc, PX[c * d + j], PL[j], PU[j]);
        out[c] = (P == 1) ? acc : sqrtf(acc / (float)smax);
    }
}

cudaError_t launch_lbp_single(const float *cand, int64_t N, const float *U, const float *L, int n, int d, int p,
                              float *out, float *scratch, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const PartGeom g = part_geom(n, d);
    float *PX = scratch, *PU = scratch + N * (int64_t)d, *PL = PU + d;
    cudaError_t e = launch_summarize(cand, N, n, d, PX, nullptr, s);
    if (e != cudaSuccess) return e;
    e = launch_query_summary(U, L, 1, n, d, nullptr, PU, PL, 0, s);
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<int64_t>((N + 255) / 256, (int64_t)device_sm_count() * 8);
    if (p == 1) k_lbp_single<1><<<blocks, 256, 0, s>>>(PX, N, PU, PL, d, g.smax, out);
    else k_lbp_single<2><<<blocks, 256, 0, s>>>(PX, N, PU, PL, d, g.smax, out);
    return cudaGetLastError();
}

}  // namespace dtwk

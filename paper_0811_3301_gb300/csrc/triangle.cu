// Ratio of the triangle-inequality experiment of App. B:
// C(x, y, z) = DTW_p(x, z) / (DTW_p(x, y) + DTW_p(y, z)), one thread per triple.
#include "common.cuh"

namespace dtwk {

__global__ void k_triangle_ratio(const float *__restrict__ dxy, const float *__restrict__ dyz,
                                 const float *__restrict__ dxz, int64_t N, float *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float num = dxz[i], den = dxy[i] + dyz[i];
        // 0 / 0 (three series at DTW distance 0) counts as no violation
        out[i] = den > 0.0f ? num / den : (num > 0.0f ? kInf : 0.0f);
    }
}

cudaError_t launch_triangle_ratio(const float *dxy, const float *dyz, const float *dxz, int64_t N, float *out,
                                  cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((N + 255) / 256, 8 * (int64_t)device_sm_count());
    k_triangle_ratio<<<blocks, 256, 0, s>>>(dxy, dyz, dxz, N, out);
    return cudaGetLastError();
}

}  // namespace dtwk

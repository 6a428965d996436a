// Template preparation at plan time (Property 2): the flipped template
// H~(j) = h(2p - j) and the FP64 sum of |h| that bounds ||A||_2.
#include "cdv_internal.h"

namespace cdv {

__global__ void flip_kernel(const float* h, float* ht, int q1, int q2, int q3)
{
    const int n = q1 * q2 * q3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j3 = i % q3, j2 = (i / q3) % q2, j1 = i / (q2 * q3);
        ht[i] = h[((q1 - 1 - j1) * q2 + (q2 - 1 - j2)) * q3 + (q3 - 1 - j3)];
    }
}

cudaError_t launch_flip(const float* h, float* ht, int q1, int q2, int q3, cudaStream_t s)
{
    const int n = q1 * q2 * q3;
    flip_kernel<<<(n + 255) / 256, 256, 0, s>>>(h, ht, q1, q2, q3);
    return cudaGetLastError();
}

// One block, fixed order: out = sum_i |h_i| in FP64.
__global__ void abs_sum_kernel(const float* h, int64_t n, double* out)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += fabs((double)h[i]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

cudaError_t launch_abs_sum(const float* h, int64_t n, double* out, cudaStream_t s)
{
    abs_sum_kernel<<<1, 256, 0, s>>>(h, n, out);
    return cudaGetLastError();
}

}  // namespace cdv

// Measurement aid, not part of the method: the FP32 fused multiply-add rate of the GPU, against
// which the FP32 convolution engine's roofline fraction is also reported (beside the nominal
// 128 lanes x 2 flop x SMs x maximum clock).
//
// Every thread runs 8 independent FMA chains (enough to cover the FMA latency with several warps
// per scheduler) for `iters` rounds and stores their sum, so nothing is dead code.
#include "cdv_internal.h"

namespace {

__global__ void __launch_bounds__(512) fma_probe_kernel(float* out, int iters)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = 1.0f + 1e-3f * (float)(tid + k);
    const float b = 0.999f, c = 1e-4f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) s += a[k];
    out[tid] = s;
}

}  // namespace

extern "C" cdv_status cdv_probe_fp32_fma(float* out, int blocks, int threads, int iters, void* stream)
{
    if (!out || blocks < 1 || threads < 32 || threads > 512 || (threads & 31) || iters < 1) {
        cdv::set_last_error("cdv_probe_fp32_fma: out != NULL, blocks >= 1, threads in {32, ..., 512} (warps), iters >= 1");
        return CDV_ERR_INVALID_ARG;
    }
    fma_probe_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(out, iters);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        cdv::set_last_error(cudaGetErrorString(e));
        return CDV_ERR_CUDA;
    }
    return CDV_OK;
}

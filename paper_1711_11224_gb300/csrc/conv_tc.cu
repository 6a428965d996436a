// Host side of the tensor-core engine (the kernel is in conv_tc.cuh): launch setup and dispatch,
// Toeplitz tiles of the template, shadow copies.  The instantiations with the step-rule variants
// live in conv_tc_var.cu so that the two sets compile in parallel.
#include "conv_tc.cuh"

namespace cdv {

size_t tc_smem_bytes(const TcArgs& t) { return TcSmem::make(t).total + 1024; }

cudaError_t tc_prepare_var(int kind);
cudaError_t tc_launch_var(const TcArgs& t, const CUtensorMap* maps, cudaStream_t s);


cudaError_t tc_prepare(int kind)
{
    cudaError_t e = tc_prepare_kinds<false>(kind);
    if (e == cudaSuccess) e = tc_prepare_var(kind);
    return e == cudaSuccess ? tc4_prepare(kind) : e;
}

// maps: 4 tensor maps (copy 0: hi0 lo0 hi1 lo1), 8 for the narrow kernel (then copy 1)
cudaError_t tc_launch(const TcArgs& t, const CUtensorMap* maps, cudaStream_t s)
{
    if (t.w4) return tc4_launch(t, maps, s);
    if ((t.W != 8 && t.W != 16) || t.P * t.W != kNT) return cudaErrorInvalidValue;
    if (t.var) return tc_launch_var(t, maps, s);
    return tc_launch_kinds<false>(t, maps, s);
}

// Toeplitz tiles T_{j1,j2}[k, n] = w[j1, j2, n + D - k] (zero outside [0, q3)),
// stored K-major for the MMA with the tiles of all j1 side by side along N, in
// groups of 8 N rows: part p, row j2, group (j1, n / 8), K chunk c, row n % 8,
// 16 bytes (EPT elements of K).  The tiles of consecutive j1 for one j2 -- one
// ring stage -- are then a single contiguous run.
__global__ void tc_btiles_kernel(const float* w, int q1, int q2, int q3, int D, int K, int W, int kind,
                                 unsigned char* hi, unsigned char* lo)
{
    const int ept = (kind == CDV_MODE_TF32) ? 4 : 8;
    const int kch = K / ept;
    const int64_t total = (int64_t)q1 * q2 * W * K;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % K);
        const int n = (int)((i / K) % W);
        const int64_t jj = i / ((int64_t)K * W);                   // j1 * q2 + j2
        const int j1 = (int)(jj / q2), j2 = (int)(jj % q2);
        const int j3 = n + D - k;
        const float v = (j3 >= 0 && j3 < q3) ? w[jj * q3 + j3] : 0.f;
        // group of 8 N rows (j1, n / 8) of template row j2, then K chunk, then the row within the group
        const size_t grp = ((size_t)j2 * q1 + j1) * (W / 8) + n / 8;
        const size_t row = (grp * kch + k / ept) * 8 + n % 8;
        const size_t off = row * 16 + (size_t)(k % ept) * (kind == CDV_MODE_TF32 ? 4 : 2);
        if (kind == CDV_MODE_TF32) {
            unsigned t;
            asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(t) : "f"(v));
            *reinterpret_cast<unsigned*>(hi + off) = t;
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
            if (kind == CDV_MODE_SPLIT_BF16X3)
                *reinterpret_cast<__nv_bfloat16*>(lo + off) = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

cudaError_t tc_build_btiles(const float* w, int q1, int q2, int q3, int D, int K, int W, int kind, void* hi, void* lo,
                            cudaStream_t s)
{
    const int64_t total = (int64_t)q1 * q2 * W * K;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    tc_btiles_kernel<<<blocks, 256, 0, s>>>(w, q1, q2, q3, D, K, W, kind, (unsigned char*)hi, (unsigned char*)lo);
    return cudaGetLastError();
}

// Shadow copy of a dense FP32 volume (a1 x a2 x a3) into the padded layout (row pitch `pitch`).
__global__ void tc_shadow_kernel(const float* src, int64_t a1a2, int64_t a3, int64_t pitch, int kind, void* hi, void* lo)
{
    const int64_t n = a1a2 * a3;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / a3, c = i - r * a3;
        const int64_t j = r * pitch + c;
        const float v = src[i];
        if (kind == CDV_MODE_TF32) {
            unsigned t;
            asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(t) : "f"(v));
            reinterpret_cast<unsigned*>(hi)[j] = t;
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            reinterpret_cast<__nv_bfloat16*>(hi)[j] = h;
            if (kind == CDV_MODE_SPLIT_BF16X3)
                reinterpret_cast<__nv_bfloat16*>(lo)[j] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

cudaError_t tc_shadow(const float* src, int64_t a1a2, int64_t a3, int64_t pitch, int kind, void* hi, void* lo,
                      cudaStream_t s)
{
    const int64_t n = a1a2 * a3;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    tc_shadow_kernel<<<blocks, 256, 0, s>>>(src, a1a2, a3, pitch, kind, hi, lo);
    return cudaGetLastError();
}

}  // namespace cdv

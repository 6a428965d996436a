// Template gradient dH(j) = sum_b sum_k X_b(k) dY_b(k + j).
//
// With Y = X (*) H, y is linear in h and dL/dh(j) = sum_k x(k) dY(k + j): the
// sum of Property 2 with the roles of x and h exchanged.  The output has only
// prod(2p+1) samples but each is a sum over every voxel of every volume, so
// the work is split over (template plane j1, chunk of voxel tiles):
//  * CTA (j1, ch) walks the tiles ch, ch + NCH, ... of (volume, plane k1, rows
//    k2, columns k3); it stages the X tile and the dY tile of plane k1 + j1
//    (rows + q2 - 1, columns + q3 - 1) in shared memory.
//  * A thread owns one template row j2 and 4 consecutive j3 for a subset of
//    the tile's rows; each 16-column block costs 4+5 16-byte shared loads for
//    64 FFMA.  Tile sums are FP32 (<= 1024 terms), accumulated across tiles
//    in FP64.
//  * Partials per (j1, ch) go to the workspace; a second kernel sums them in
//    FP64 in chunk order (deterministic, no atomics).
#include <algorithm>

#include "cdv_internal.h"

namespace cdv {

namespace {
constexpr int KC = 16;      // rows (axis 2) per tile
constexpr int KW = 64;      // columns (axis 3) per tile
constexpr int RJ = 4;       // j3 values per thread

struct GLayout {
    int nj3, S, threads, drows, dpitch;
    static GLayout make(const GradPsfPlan& g)
    {
        GLayout l;
        l.nj3 = (g.q3 + RJ - 1) / RJ;
        const int per = g.q2 * l.nj3;
        l.S = std::max(1, std::min(KC, 256 / std::max(1, per)));
        l.threads = l.S * per;
        l.drows = KC + g.q2 - 1;
        l.dpitch = ((KW + RJ * l.nj3 + 3) & ~3) + 4;
        return l;
    }
};
}  // namespace

size_t grad_psf_partials(const GradPsfPlan& g) { return (size_t)g.q1 * g.chunks * g.q2 * g.q3; }

__device__ __forceinline__ void cpa4(float* dst, const float* src, bool ok)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}

__global__ void __launch_bounds__(1024) grad_psf_kernel(GradPsfPlan g, GLayout l, const float* X, const float* dY,
                                                        double* partial)
{
    extern __shared__ __align__(16) float sm[];
    float* s_x = sm;                                  // KC x KW
    float* s_d = sm + KC * KW;                        // drows x dpitch
    double* s_red = reinterpret_cast<double*>(s_d + l.drows * l.dpitch + ((l.drows * l.dpitch) & 1));

    const int j1 = blockIdx.x / g.chunks, ch = blockIdx.x % g.chunks;
    const int tid = threadIdx.x;
    const int per = g.q2 * l.nj3;
    const int js = tid / per, rem = tid % per;
    const int j2 = rem / l.nj3, jg = rem % l.nj3;
    const bool active = tid < l.threads;

    const int64_t n2 = g.m2 + g.q2 - 1, n3 = g.m3 + g.q3 - 1, n1 = g.m1 + g.q1 - 1;
    const int64_t t2 = (g.m2 + KC - 1) / KC, t3 = (g.m3 + KW - 1) / KW;
    const int64_t ntiles = (int64_t)g.batch * g.m1 * t2 * t3;

    double dacc[RJ] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t t = ch; t < ntiles; t += g.chunks) {
        int64_t r = t;
        const int64_t i3 = r % t3; r /= t3;
        const int64_t i2 = r % t2; r /= t2;
        const int64_t k1 = r % g.m1;
        const int64_t b = r / g.m1;
        const int64_t K2 = i2 * KC, K3 = i3 * KW;
        const float* xp = X + (b * g.m1 + k1) * g.m2 * g.m3;
        const float* dp = dY + (b * n1 + (k1 + j1)) * n2 * n3;
        for (int e = tid; e < KC * KW; e += blockDim.x) {
            const int rr = e / KW, cc = e % KW;
            const int64_t k2 = K2 + rr, k3 = K3 + cc;
            const bool ok = k2 < g.m2 && k3 < g.m3;
            cpa4(s_x + e, ok ? xp + k2 * g.m3 + k3 : X, ok);
        }
        for (int e = tid; e < l.drows * l.dpitch; e += blockDim.x) {
            const int rr = e / l.dpitch, cc = e % l.dpitch;
            const int64_t v = K2 + rr, c = K3 + cc;
            const bool ok = v < n2 && c < n3;
            cpa4(s_d + e, ok ? dp + v * n3 + c : dY, ok);
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        if (active) {
            float acc[RJ] = {0.f, 0.f, 0.f, 0.f};
            for (int rr = js; rr < KC; rr += l.S) {
                const float* xr = s_x + rr * KW;
                const float* dr = s_d + (rr + j2) * l.dpitch + RJ * jg;
#pragma unroll 2
                for (int kb = 0; kb < KW; kb += 16) {
                    float xv[16], dv[20];
#pragma unroll
                    for (int i = 0; i < 16; i += 4) {
                        const float4 a = *reinterpret_cast<const float4*>(xr + kb + i);
                        xv[i] = a.x; xv[i + 1] = a.y; xv[i + 2] = a.z; xv[i + 3] = a.w;
                    }
#pragma unroll
                    for (int i = 0; i < 20; i += 4) {
                        const float4 a = *reinterpret_cast<const float4*>(dr + kb + i);
                        dv[i] = a.x; dv[i + 1] = a.y; dv[i + 2] = a.z; dv[i + 3] = a.w;
                    }
#pragma unroll
                    for (int i = 0; i < 16; i++)
#pragma unroll
                        for (int q = 0; q < RJ; q++) acc[q] = fmaf(xv[i], dv[i + q], acc[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < RJ; q++) dacc[q] += (double)acc[q];
        }
        __syncthreads();
    }
    // reduce over the row subsets js in a fixed order
    if (active)
#pragma unroll
        for (int q = 0; q < RJ; q++) s_red[tid * RJ + q] = dacc[q];
    __syncthreads();
    if (active && js == 0) {
        for (int q = 0; q < RJ; q++) {
            const int j3 = RJ * jg + q;
            if (j3 >= g.q3) continue;
            double s = 0.0;
            for (int k = 0; k < l.S; k++) s += s_red[(k * per + rem) * RJ + q];
            partial[((int64_t)j1 * g.chunks + ch) * g.q2 * g.q3 + j2 * g.q3 + j3] = s;
        }
    }
}

__global__ void grad_psf_final_kernel(GradPsfPlan g, const double* partial, float* dH)
{
    const int n = g.q1 * g.q2 * g.q3;
    const int per = g.q2 * g.q3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j1 = i / per, r = i % per;
        double s = 0.0;
        for (int c = 0; c < g.chunks; c++) s += partial[((int64_t)j1 * g.chunks + c) * per + r];
        dH[i] = (float)s;
    }
}

cudaError_t grad_psf_prepare()
{
    return cudaFuncSetAttribute(grad_psf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradPsfMaxSmem);
}

size_t grad_psf_smem_bytes(const GradPsfPlan& g)
{
    const GLayout l = GLayout::make(g);
    if (l.threads > 1024) return 0;
    const int threads = (l.threads + 31) & ~31;
    size_t fl = (size_t)KC * KW + (size_t)l.drows * l.dpitch;
    fl = (fl + 1) & ~(size_t)1;
    return fl * sizeof(float) + (size_t)threads * RJ * sizeof(double);
}

cudaError_t launch_grad_psf(const GradPsfPlan& g, const float* X, const float* dY, double* partial, float* dH,
                            cudaStream_t s)
{
    const GLayout l = GLayout::make(g);
    const size_t smem = grad_psf_smem_bytes(g);
    if (smem == 0 || smem > kGradPsfMaxSmem) return cudaErrorInvalidConfiguration;
    const int threads = (l.threads + 31) & ~31;
    grad_psf_kernel<<<g.q1 * g.chunks, threads, smem, s>>>(g, l, X, dY, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n = g.q1 * g.q2 * g.q3;
    grad_psf_final_kernel<<<(n + 255) / 256, 256, 0, s>>>(g, partial, dH);
    return cudaGetLastError();
}

}  // namespace cdv

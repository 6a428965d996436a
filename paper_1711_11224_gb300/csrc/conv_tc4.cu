// Host side of the narrow tensor-core kernel (conv_tc4.cuh): launch, template stages, shifted
// shadow copies.  The instantiations with the step-rule variants are in conv_tc4_var.cu.
#include <vector>

#include "conv_tc4.cuh"

namespace cdv {

size_t tc4_smem_bytes(const TcArgs& t) { return Tc4Smem::make(t).total + 1024; }

size_t tc4_btiles_bytes(const TcArgs& t) { return (size_t)t.nst * 2 * kSlots * (2 * t.spst) * 128; }

cudaError_t tc4_prepare_var(int kind);
cudaError_t tc4_launch_var(const TcArgs& t, const CUtensorMap* maps, cudaStream_t s);

cudaError_t tc4_prepare(int kind)
{
    cudaError_t e = tc4_prepare_kinds<false>(kind);
    return e == cudaSuccess ? tc4_prepare_var(kind) : e;
}

cudaError_t tc4_launch(const TcArgs& t, const CUtensorMap* maps, cudaStream_t s)
{
    if (!t.w4 || t.kc < 1 || t.spst != t.kc || t.nst * t.spst < t.steps) return cudaErrorInvalidValue;
    if (t.var) return tc4_launch_var(t, maps, s);
    return tc4_launch_kinds<false>(t, maps, s);
}

// Template stages of the narrow kernel, per part: [stage t][version v][group e][chunk cc][row n8][8 elements].
// Group e of version v holds the Toeplitz tiles of doubled-sequence entries i = 2e + v and 2e + v + 1
// (template plane i mod 32; plane 31 and planes >= q1 are zero), 4 N rows each: row n8 is column
// n8 % 4 of entry n8 / 4.  Chunk cc of stage t is the first (even cc) or second (odd cc) chunk of
// K step t * spst + cc / 2, in the order tc4_step gives; its 8 elements are window columns
// 8c .. 8c + 7 of template row j2, and T[k, n] = w[j1, j2, n + q3 - 1 - k].
__global__ void tc4_btiles_kernel(const float* w, int q1, int q2, int q3, int kc, int rows, int steps, int spst,
                                  int64_t total, int kind, __nv_bfloat16* hi, __nv_bfloat16* lo)
{
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = idx;
        const int e = (int)(r % 8); r /= 8;
        const int n8 = (int)(r % 8); r /= 8;
        const int cc = (int)(r % (2 * spst)); r /= 2 * spst;
        const int grp = (int)(r % kSlots); r /= kSlots;
        const int ver = (int)(r % 2);
        const int t = (int)(r / 2);
        float v = 0.f;
        const int step = t * spst + cc / 2;
        if (step < steps) {
            const StepA sa = tc4_step(step, q2, kc, rows);
            const int item = (cc & 1) ? sa.second : sa.first;
            if (item < q2 * kc) {
                const int j1 = (2 * grp + ver + n8 / 4) % kSlots;
                const int j2 = item / kc, c = item % kc;
                const int j3 = (n8 % 4) + q3 - 1 - (8 * c + e);
                if (j1 < q1 && j3 >= 0 && j3 < q3) v = w[((int64_t)j1 * q2 + j2) * q3 + j3];
            }
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[idx] = h;
        if (kind == CDV_MODE_SPLIT_BF16X3) lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

cudaError_t tc4_build_btiles(const TcArgs& t, const float* w, void* hi, void* lo, cudaStream_t s)
{
    const int64_t total = (int64_t)tc4_btiles_bytes(t) / 2;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    tc4_btiles_kernel<<<blocks, 256, 0, s>>>(w, t.g.q1, t.g.q2, t.g.q3, t.kc, t.rows, t.steps, t.spst, total, t.kind,
                                             (__nv_bfloat16*)hi, (__nv_bfloat16*)lo);
    return cudaGetLastError();
}

// The shifted shadow copy: row r of a dense FP32 volume (a1 a2 rows of a3) goes to columns 4 .. a3 + 3
// of row r (pitch1 elements); columns 0-3 keep the zeros the plan wrote once.
__global__ void tc4_shadow1_kernel(const float* src, int64_t a1a2, int64_t a3, int64_t pitch1, int kind,
                                   __nv_bfloat16* hi, __nv_bfloat16* lo)
{
    const int64_t n = a1a2 * a3;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / a3, c = i - r * a3;
        const int64_t j = r * pitch1 + c + 4;
        const float v = src[i];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[j] = h;
        if (kind == CDV_MODE_SPLIT_BF16X3) lo[j] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

cudaError_t tc4_shadow1(const float* src, int64_t a1a2, int64_t a3, int64_t pitch1, int kind, void* hi, void* lo,
                        cudaStream_t s)
{
    const int64_t n = a1a2 * a3;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    tc4_shadow1_kernel<<<blocks, 256, 0, s>>>(src, a1a2, a3, pitch1, kind, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo);
    return cudaGetLastError();
}

}  // namespace cdv

namespace cdv {

// Tensor-pipe work of one launch of the narrow kernel, counting its loops: per tile and input plane,
// `steps` MMAs of K = 16 and N = 4 x (slots covered) for each 128-row M tile holding outputs.
double tc4_executed_macs(const TcArgs& t)
{
    const ConvGeom& g = t.g;
    double macs = 0.0;
    for (int tile = 0; tile < t.ntiles; tile++) {
        const Tc4Tile C = Tc4Tile::make(t, tile);
        const int64_t nmt = std::min<int64_t>(kMT, (g.b2 - C.S2 + kM - 1) / kM);
        for (int64_t u = C.ulo; u <= C.uhi; u++) {
            int k0, ns;
            C.mma_slots(g, u, k0, ns);
            macs += (double)t.steps * 16.0 * (double)(kW4 * ns) * (double)(kM * nmt);
        }
    }
    return macs * ((t.nprec == 2) ? 3.0 : 1.0);
}

// Modelled tensor-pipe cycles of one launch: each MMA costs about max(46, N / 2) cycles, and the
// persistent CTAs take tiles blockIdx.x, blockIdx.x + grid, ... (the slowest CTA sets the time).
double tc4_model_cycles(const TcArgs& t)
{
    const ConvGeom& g = t.g;
    std::vector<double> cta(std::max(1, t.grid), 0.0);
    for (int tile = 0; tile < t.ntiles; tile++) {
        const Tc4Tile C = Tc4Tile::make(t, tile);
        const int64_t nmt = std::min<int64_t>(kMT, (g.b2 - C.S2 + kM - 1) / kM);
        double c = 0.0;
        for (int64_t u = C.ulo; u <= C.uhi; u++) {
            int k0, ns;
            C.mma_slots(g, u, k0, ns);
            c += std::max(46.0, kW4 * ns / 2.0);
        }
        cta[tile % cta.size()] += c * t.steps * (double)nmt;
    }
    return *std::max_element(cta.begin(), cta.end());
}

}  // namespace cdv

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
    if (!t.w4 || t.kc < 1 || t.spst < 1 || t.na != 2 || t.nst * t.spst < t.steps || !t.tlist || !t.toff)
        return cudaErrorInvalidValue;
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

// Farthest column (exclusive) that the window loads of a direction's tiles reach in each shadow copy:
// column group g reads kc chunks from x = 4g + o3 - (q3 - 1), in copy 0 when x is a multiple of 8, else
// in copy 1 (shifted right by 4 columns) from x + 4.
void tc4_window_extent(const TcArgs& t, int64_t need[2])
{
    const ConvGeom& g = t.g;
    need[0] = need[1] = 0;
    for (int64_t s3 = 0; s3 < g.b3; s3 += kW4) {
        const int64_t x = s3 + g.o3 - (g.q3 - 1);
        const int c = (((x % 8) + 8) % 8) == 0 ? 0 : 1;
        need[c] = std::max(need[c], x + 4 * c + 8 * (int64_t)t.kc);
    }
    if (t.flat && t.nblk > 0) {
        // the last M block also stages rows past the last group (they hold no outputs), read from copy 1
        const int64_t last = (int64_t)(t.nblk - 1) * kM * kMT + t.fboxes * 32 - 1;
        const int64_t gl = last / t.lp - t.ngrp[0];
        const int64_t x0 = 4 * (int64_t)t.gfirst[1] + g.o3 - (g.q3 - 1) + 4;
        if (gl >= 0) need[1] = std::max(need[1], x0 + 8 * gl + 8 * (int64_t)t.kc);
    }
}

// Weight of a tile's M tiles in the cycle model: a plane with one 128-row M tile costs about 0.67 of a
// plane with two (measured per CTA on ring3d's forward), not half: the template stages and input boxes
// of a plane are the same for one or two M tiles.
static double tc4_mt_weight(int nmt) { return nmt == 1 ? 1.35 : (double)nmt; }

// Modelled tensor-pipe cycles of the MMAs of one tile: each MMA costs about max(46, N / 2) cycles.
static double tc4_tile_cycles(const TcArgs& t, const Tc4Tile& C)
{
    double c = 0.0;
    for (int64_t u = C.ulo; u <= C.uhi; u++) {
        int k0, ns;
        C.mma_slots(t.g, u, k0, ns);
        c += std::max(46.0, kW4 * ns / 2.0);
    }
    return c * t.steps * tc4_mt_weight(C.mtiles(t));
}

// Tensor-pipe work of one launch of the narrow kernel, counting its loops: per tile and input plane,
// `steps` MMAs of K = 16 and N = 4 x (slots covered) for each 128-row M tile holding outputs.
double tc4_executed_macs(const TcArgs& t, const std::vector<int4>& list)
{
    double macs = 0.0;
    for (const int4& d : list) {
        const Tc4Tile C = Tc4Tile::make(t, d);
        for (int64_t u = C.ulo; u <= C.uhi; u++) {
            int k0, ns;
            C.mma_slots(t.g, u, k0, ns);
            macs += (double)t.steps * 16.0 * (double)(kW4 * ns) * (double)(kM * C.mtiles(t));
        }
    }
    return macs * ((t.nprec == 2) ? 3.0 : 1.0);
}

// Tile lists of the persistent CTAs, dealt out in order under a load bound T (the smallest, by binary
// search on the cycle model, for which nsm CTAs suffice):
//  * pc = 0: M block (combo) by M block, each block's b1 output planes cut into 32-aligned ranges as
//    long as the CTA's bound allows (long ranges waste less at the plane-chunk ends, where an input
//    plane reaches few slots);
//  * pc > 0: chunks of pc planes, all M blocks of a chunk before the next chunk, so that the CTAs
//    running at the same time read the same input planes (shared through L2).
double tc4_partition(TcArgs& t, int nsm, int pc, std::vector<int4>& list, std::vector<int>& off)
{
    const ConvGeom& g = t.g;
    const int ncombo = t.flat ? t.nblk : t.tiles2 * t.tiles3;
    const int nb = (int)((g.b1 + 31) / 32);                  // 32-plane units
    // cycles of planes [32a, min(32e, b1)) of a combo with one M tile (a < e), cached
    std::vector<double> cost((size_t)nb * (nb + 1), -1.0);
    auto chunk = [&](int a, int e) {
        double& c = cost[(size_t)a * (nb + 1) + e];
        if (c < 0.0) {
            TcArgs one = t;
            one.flat = 0;
            one.tiles2 = 1;
            one.tiles3 = 1;
            const Tc4Tile C = Tc4Tile::make(one, make_int4(32 * a, (int)std::min<int64_t>(32 * (int64_t)e, g.b1), 0, 0));
            // one M tile of outputs (S2 = 0 with b2 of at least one row): scaled by the combo's M tiles below
            c = tc4_tile_cycles(one, C) / tc4_mt_weight(std::max(1, C.mtiles(one)));
        }
        return c;
    };
    std::vector<double> nmt(ncombo);
    for (int j = 0; j < ncombo; j++) nmt[j] = tc4_mt_weight(Tc4Tile::make(t, make_int4(0, (int)g.b1, j, 0)).mtiles(t));
    auto deal = [&](double T, std::vector<int4>* L, std::vector<int>* O) -> int {
        int cta = 0;
        double load = 0.0;
        if (O) O->assign(1, 0);
        if (pc > 0) {
            const int pu = pc / 32;
            for (int a = 0; a < nb; a += pu)
                for (int j = 0; j < ncombo; j++) {
                    const int e = std::min(nb, a + pu);
                    const double c = chunk(a, e) * nmt[j];
                    if (load > 0.0 && load + c > T) {
                        if (O) O->push_back((int)L->size());
                        cta++;
                        load = 0.0;
                    }
                    if (c > T) return 1 << 30;
                    if (L) L->push_back(make_int4(32 * a, (int)std::min<int64_t>(32 * (int64_t)e, g.b1), j, 0));
                    load += c;
                }
            if (O) O->push_back((int)L->size());
            return cta + 1;
        }
        for (int j = 0; j < ncombo; j++) {
            int a = 0;
            while (a < nb) {
                int e = a;
                while (e < nb && load + chunk(a, e + 1) * nmt[j] <= T) e++;
                if (e == a) {
                    if (load == 0.0) return 1 << 30;             // one 32-plane tile exceeds T
                    if (O) O->push_back((int)L->size());
                    cta++;
                    load = 0.0;
                    continue;
                }
                if (L) L->push_back(make_int4(32 * a, (int)std::min<int64_t>(32 * (int64_t)e, g.b1), j, 0));
                load += chunk(a, e) * nmt[j];
                a = e;
            }
        }
        if (O) O->push_back((int)L->size());
        return cta + 1;
    };
    double hi = 0.0;
    for (int j = 0; j < ncombo; j++) hi += chunk(0, nb) * nmt[j];
    double lo = 0.0;
    for (int it = 0; it < 60 && hi - lo > 1e-4 * hi; it++) {
        const double mid = 0.5 * (lo + hi);
        if (deal(mid, nullptr, nullptr) <= nsm) hi = mid;
        else lo = mid;
    }
    list.clear();
    deal(hi, &list, &off);
    t.grid = (int)off.size() - 1;
    t.ntiles = (int)list.size();
    double mk = 0.0;
    for (int b = 0; b < t.grid; b++) {
        double c = 0.0;
        for (int k = off[b]; k < off[b + 1]; k++) c += tc4_tile_cycles(t, Tc4Tile::make(t, list[k]));
        mk = std::max(mk, c);
    }
    return mk;
}

}  // namespace cdv

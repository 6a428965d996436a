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

// Narrow templates (q3 <= 15): a register-blocked form with double-buffered 16-byte staging.
//  * CTA (j1, ch) walks tiles (volume, plane k1, rows k2 .. k2 + 15, columns k3 .. k3 + 63);
//    thread (jp, rs) owns all Q3 outputs dH(j1, j2, .) of template rows j2 = jp and jp + ceil(q2 / 2)
//    (so the dY rows that the threads of a quarter warp read lie within 8 consecutive rows: no bank
//    conflicts, where rows 2 jp and 2 jp + 1 put rows 8 apart on the same banks) for the tile rows
//    rs, rs + RS, ...
//  * Per 8 columns of a row: two 16-byte loads of x, 2 ceil((Q3 + 7) / 4) of the dY rows k2 + j2, and
//    16 Q3 FMAs (Q3 + 7 window values against 8 x values, for both rows j2).
//  * The next tile is copied (cp.async) while the current one is summed; sums are FP32 over as many
//    tiles as keep them at 1024 terms per thread at most, then added into FP64 sums (shared memory),
//    which are reduced over rs in a fixed order.
//  * One wave: q1 x chunks CTAs fill every SM's resident slots once (grad_psf_chunks).
constexpr int QKW = 64;             // columns per tile
constexpr int QTR = 16;             // rows per tile

// Row pitches in floats, an odd number of 16-byte units: the rows that the threads of a warp read at one
// column (different j2 and row subsets) then fall on different banks.
constexpr int QXP = QKW + 4;
template <int Q3>
struct QLayout {
    static constexpr int DW = ((QKW + Q3 + 3 + 3) / 4) * 4;               // window read per row
    static constexpr int DP = ((DW / 4) & 1) ? DW : DW + 4;               // dY tile pitch
};

__device__ __forceinline__ void cpa16(float* dst, const float* src, int bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}

template <int Q3>
__global__ void __launch_bounds__(512) grad_psf_q_kernel(GradPsfPlan g, int RS, bool vec, const float* X,
                                                         const float* dY, double* partial)
{
    constexpr int DP = QLayout<Q3>::DP;
    constexpr int NW8 = (Q3 + 7 + 3) / 4;                   // 16-byte loads of one dY window of 8 columns
    extern __shared__ __align__(16) float smq[];
    const int q2 = g.q2, drows = QTR + q2 - 1, npair = (q2 + 1) / 2;
    const int buf = QTR * QXP + drows * DP;                 // floats per buffer
    double* s_acc = reinterpret_cast<double*>(smq + 2 * buf);   // FP64 sums across tiles, [tid][2][Q3]
    const int j1 = blockIdx.x / g.chunks, ch = blockIdx.x % g.chunks;
    const int tid = threadIdx.x, nthr = npair * RS;
    const int jp = tid % npair, rs = tid / npair;
    const int j2a = jp, j2b = min(jp + npair, q2 - 1);      // a lone last row is summed twice, kept once
    const bool active = tid < nthr;
    const int64_t n2 = g.m2 + g.q2 - 1, n3 = g.m3 + Q3 - 1, n1 = g.m1 + g.q1 - 1;
    const int64_t t2 = (g.m2 + QTR - 1) / QTR, t3 = (g.m3 + QKW - 1) / QKW;
    const int64_t ntiles = (int64_t)g.batch * g.m1 * t2 * t3;
    if (active)
        for (int q = 0; q < 2 * Q3; q++) s_acc[tid * 2 * Q3 + q] = 0.0;

    // stage tile t into buffer b: X rows k2 .. k2 + 15 (zero outside), dY rows k2 .. k2 + drows - 1
    auto stage = [&](int64_t t, int b) {
        int64_t r = t;
        const int64_t i3 = r % t3; r /= t3;
        const int64_t i2 = r % t2; r /= t2;
        const int64_t k1 = r % g.m1;
        const int64_t bb = r / g.m1;
        const int64_t K2 = i2 * QTR, K3 = i3 * QKW;
        const float* xp = X + (bb * g.m1 + k1) * g.m2 * g.m3;
        const float* dp = dY + (bb * n1 + (k1 + j1)) * n2 * n3;
        float* sx = smq + b * buf;
        float* sd = sx + QTR * QXP;
        if (vec) {
            for (int e = tid; e < QTR * QKW / 4; e += blockDim.x) {
                const int rr = e / (QKW / 4), cc = 4 * (e % (QKW / 4));
                const int64_t k2 = K2 + rr, k3 = K3 + cc;
                const int64_t left = (k2 < g.m2) ? g.m3 - k3 : 0;
                const int bytes = left >= 4 ? 16 : (left > 0 ? (int)left * 4 : 0);
                cpa16(sx + rr * QXP + cc, bytes ? xp + k2 * g.m3 + k3 : X, bytes);
            }
            for (int e = tid; e < drows * DP / 4; e += blockDim.x) {
                const int rr = e / (DP / 4), cc = 4 * (e % (DP / 4));
                const int64_t v = K2 + rr, c = K3 + cc;
                const int64_t left = (v < n2) ? n3 - c : 0;
                const int bytes = left >= 4 ? 16 : (left > 0 ? (int)left * 4 : 0);
                cpa16(sd + rr * DP + cc, bytes ? dp + v * n3 + c : dY, bytes);
            }
        } else {
            for (int e = tid; e < QTR * QKW; e += blockDim.x) {
                const int rr = e / QKW, cc = e % QKW;
                const int64_t k2 = K2 + rr, k3 = K3 + cc;
                const bool ok = k2 < g.m2 && k3 < g.m3;
                cpa4(sx + rr * QXP + cc, ok ? xp + k2 * g.m3 + k3 : X, ok);
            }
            for (int e = tid; e < drows * DP; e += blockDim.x) {
                const int rr = e / DP, cc = e % DP;
                const int64_t v = K2 + rr, c = K3 + cc;
                const bool ok = v < n2 && c < n3;
                cpa4(sd + e, ok ? dp + v * n3 + c : dY, ok);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    // FP32 sums run over `flush` tiles (at most 1024 products each: 64 columns x ceil(16 / RS) rows per
    // tile) before they are added to the FP64 sums: GB300 runs FP64 adds at a small fraction of the FP32
    // FMA rate, and adding after every tile (22 adds per 1,408 FMAs for q3 = 11, RS = 16) kept the FP64
    // pipe 61% busy against 35% for the FMAs
    const int flush = max(1, QTR / ((QTR + RS - 1) / RS));
    float acc[2][Q3];
#pragma unroll
    for (int q = 0; q < Q3; q++) acc[0][q] = acc[1][q] = 0.f;
    int nacc = 0;
    int b = 0;
    if (ch < ntiles) stage(ch, 0);
    for (int64_t t = ch; t < ntiles; t += g.chunks, b ^= 1) {
        if (t + g.chunks < ntiles) {
            stage(t + g.chunks, b ^ 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        if (active) {
            const float* sx = smq + b * buf;
            const float* sd = sx + QTR * QXP;
            for (int rr = rs; rr < QTR; rr += RS) {
                const float* xr = sx + rr * QXP;
                const float* da = sd + (rr + j2a) * DP;
                const float* db = sd + (rr + j2b) * DP;
                // 8 columns per step (two x loads and NW8 loads of each dY window for 16 Q3 FMAs), columns
                // in ascending order as four at a time would take them
#pragma unroll 1
                for (int kb = 0; kb < QKW; kb += 8) {
                    const float4 x0 = *reinterpret_cast<const float4*>(xr + kb);
                    const float4 x1 = *reinterpret_cast<const float4*>(xr + kb + 4);
                    const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                    float wa[4 * NW8], wb[4 * NW8];
#pragma unroll
                    for (int i = 0; i < NW8; i++) {
                        const float4 a = *reinterpret_cast<const float4*>(da + kb + 4 * i);
                        const float4 c = *reinterpret_cast<const float4*>(db + kb + 4 * i);
                        wa[4 * i] = a.x; wa[4 * i + 1] = a.y; wa[4 * i + 2] = a.z; wa[4 * i + 3] = a.w;
                        wb[4 * i] = c.x; wb[4 * i + 1] = c.y; wb[4 * i + 2] = c.z; wb[4 * i + 3] = c.w;
                    }
#pragma unroll
                    for (int e = 0; e < 8; e++)
#pragma unroll
                        for (int q = 0; q < Q3; q++) {
                            acc[0][q] = fmaf(xv[e], wa[q + e], acc[0][q]);
                            acc[1][q] = fmaf(xv[e], wb[q + e], acc[1][q]);
                        }
                }
            }
            if (++nacc == flush || t + g.chunks >= ntiles) {
                double* sa = s_acc + tid * 2 * Q3;
#pragma unroll
                for (int q = 0; q < Q3; q++) {
                    sa[q] += (double)acc[0][q];
                    sa[Q3 + q] += (double)acc[1][q];
                    acc[0][q] = acc[1][q] = 0.f;
                }
                nacc = 0;
            }
        }
        __syncthreads();                                   // buffer b is overwritten by the next stage
    }
    // reduce over the row subsets rs in a fixed order
    __syncthreads();
    if (active && rs == 0) {
        for (int h = 0; h < 2; h++) {
            const int j2 = h ? jp + npair : jp;
            if (j2 >= q2) continue;
            for (int q = 0; q < Q3; q++) {
                double sum = 0.0;
                for (int k = 0; k < RS; k++) sum += s_acc[(k * npair + jp) * 2 * Q3 + h * Q3 + q];
                partial[((int64_t)j1 * g.chunks + ch) * g.q2 * Q3 + j2 * Q3 + q] = sum;
            }
        }
    }
}

// Row subsets per CTA of the narrow form: ceil(q2 / 2) x RS threads (at most 512), RS <= 16 (a tile has
// 16 rows).
static int grad_q_rs(const GradPsfPlan& g) { return std::max(1, std::min(QTR, 512 / std::max(1, (g.q2 + 1) / 2))); }

template <int Q3>
static size_t grad_q_smem(const GradPsfPlan& g)
{
    const int drows = QTR + g.q2 - 1;
    const size_t buf = (size_t)QTR * QXP + (size_t)drows * QLayout<Q3>::DP;
    return 2 * buf * sizeof(float) + (size_t)((g.q2 + 1) / 2) * grad_q_rs(g) * 2 * Q3 * sizeof(double);
}

template <int Q3>
static cudaError_t launch_grad_q(const GradPsfPlan& g, const float* X, const float* dY, double* partial, cudaStream_t s)
{
    const int RS = grad_q_rs(g);
    const size_t smem = grad_q_smem<Q3>(g);
    const bool vec = (g.m3 % 4 == 0) && ((g.m3 + Q3 - 1) % 4 == 0) && ((uintptr_t)X % 16 == 0) && ((uintptr_t)dY % 16 == 0);
    const int threads = (((g.q2 + 1) / 2) * RS + 31) & ~31;
    grad_psf_q_kernel<Q3><<<g.q1 * g.chunks, threads, smem, s>>>(g, RS, vec, X, dY, partial);
    return cudaGetLastError();
}

template <int Q3>
static cudaError_t prepare_grad_q()
{
    return cudaFuncSetAttribute(grad_psf_q_kernel<Q3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradPsfMaxSmem);
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
    cudaError_t e = cudaFuncSetAttribute(grad_psf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradPsfMaxSmem);
    if (e == cudaSuccess) e = prepare_grad_q<1>();
    if (e == cudaSuccess) e = prepare_grad_q<3>();
    if (e == cudaSuccess) e = prepare_grad_q<5>();
    if (e == cudaSuccess) e = prepare_grad_q<7>();
    if (e == cudaSuccess) e = prepare_grad_q<9>();
    if (e == cudaSuccess) e = prepare_grad_q<11>();
    if (e == cudaSuccess) e = prepare_grad_q<13>();
    if (e == cudaSuccess) e = prepare_grad_q<15>();
    return e;
}

// The narrow form applies to q3 <= 15 with at most 512 threads of template rows and its shared memory.
static bool grad_q_ok(const GradPsfPlan& g)
{
    if (g.q3 > 15 || g.q3 < 1 || !(g.q3 & 1) || g.q2 > 1024) return false;
    size_t smem = 0;
    switch (g.q3) {
    case 1: smem = grad_q_smem<1>(g); break;
    case 3: smem = grad_q_smem<3>(g); break;
    case 5: smem = grad_q_smem<5>(g); break;
    case 7: smem = grad_q_smem<7>(g); break;
    case 9: smem = grad_q_smem<9>(g); break;
    case 11: smem = grad_q_smem<11>(g); break;
    case 13: smem = grad_q_smem<13>(g); break;
    default: smem = grad_q_smem<15>(g); break;
    }
    return smem <= kGradPsfMaxSmem;
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

// Chunks of the voxel tiles per template plane: for the narrow form one full wave of resident CTAs
// (q1 x chunks = CTAs per SM x SMs), so that no second, nearly empty wave of long CTAs remains.
template <int Q3>
static int grad_q_chunks(const GradPsfPlan& g)
{
    int per_sm = 0, dev = 0, nsm = 0;
    const int RS = grad_q_rs(g);
    const int threads = (((g.q2 + 1) / 2) * RS + 31) & ~31;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grad_psf_q_kernel<Q3>, threads, grad_q_smem<Q3>(g)) !=
            cudaSuccess ||
        per_sm < 1)
        return std::max(1, (152 * 4 + g.q1 - 1) / g.q1);
    return std::max(1, per_sm * nsm / g.q1);
}

int grad_psf_chunks(const GradPsfPlan& g)
{
    if (!grad_q_ok(g)) return std::max(1, (152 * 4 + g.q1 - 1) / g.q1);
    switch (g.q3) {
    case 1: return grad_q_chunks<1>(g);
    case 3: return grad_q_chunks<3>(g);
    case 5: return grad_q_chunks<5>(g);
    case 7: return grad_q_chunks<7>(g);
    case 9: return grad_q_chunks<9>(g);
    case 11: return grad_q_chunks<11>(g);
    case 13: return grad_q_chunks<13>(g);
    default: return grad_q_chunks<15>(g);
    }
}

cudaError_t launch_grad_psf(const GradPsfPlan& g, const float* X, const float* dY, double* partial, float* dH,
                            cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (grad_q_ok(g)) {
        switch (g.q3) {
        case 1: e = launch_grad_q<1>(g, X, dY, partial, s); break;
        case 3: e = launch_grad_q<3>(g, X, dY, partial, s); break;
        case 5: e = launch_grad_q<5>(g, X, dY, partial, s); break;
        case 7: e = launch_grad_q<7>(g, X, dY, partial, s); break;
        case 9: e = launch_grad_q<9>(g, X, dY, partial, s); break;
        case 11: e = launch_grad_q<11>(g, X, dY, partial, s); break;
        case 13: e = launch_grad_q<13>(g, X, dY, partial, s); break;
        default: e = launch_grad_q<15>(g, X, dY, partial, s); break;
        }
    } else {
        const GLayout l = GLayout::make(g);
        const size_t smem = grad_psf_smem_bytes(g);
        if (smem == 0 || smem > kGradPsfMaxSmem) return cudaErrorInvalidConfiguration;
        const int threads = (l.threads + 31) & ~31;
        grad_psf_kernel<<<g.q1 * g.chunks, threads, smem, s>>>(g, l, X, dY, partial);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    const int n = g.q1 * g.q2 * g.q3;
    grad_psf_final_kernel<<<(n + 255) / 256, 256, 0, s>>>(g, partial, dH);
    return cudaGetLastError();
}

}  // namespace cdv

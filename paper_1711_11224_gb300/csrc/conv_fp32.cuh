// FP32 direct-convolution engine on the CUDA cores.
//
// Computes, for every output sample s of a 3-D box,
//     out[s] = sum_{j in [0,q)} w[j] * in[s + o - j]      (in = 0 outside its box)
// which is the forward operator of Property 1 (in = X, o = 0, w = H, output
// m + 2p) and the adjoint of Property 2 (in = R, o = 2p, w = H~, output m).
//
// Work decomposition (one CTA per output tile of T1 planes x nty rows x
// ntx*R3 columns; one thread per row and R3 consecutive columns, all T1
// planes):
//  * The CTA streams the input planes u that reach its output planes.  Plane
//    u's halo tile ((nty + q2 - 1) rows x pitch columns) and the T1 template
//    planes j1 = s1 + o1 - u it meets are staged in shared memory with
//    cp.async, double buffered, zero-filled outside the input box.
//  * For each template row j2 a thread loads its input window of R3+Q3-1
//    values into registers (16-byte shared loads) and slides it against the
//    Q3 taps of every valid output plane (R3*Q3 FFMA per window per plane).
//  * Two-level summation: the taps of one input plane are summed into a
//    per-plane partial that is then added to the running total.  A single
//    FP32 accumulator over all q1*q2*q3 taps loses the small terms of wide
//    templates (about 1e-5 relative at 31x31x21); per-plane partials keep
//    the error near 1e-7.
//  * Output rows whose input rows fall outside the box skip those template
//    rows (exact skipping along axes 1 and 2; along axis 3 the window is
//    zero-padded).
//  * Epilogues fuse the residual, the projected update, Richardson-Lucy
//    ratios and the FP64 block partials of the iteration's norms.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cdv_internal.h"

namespace cdv {

constexpr int kR3 = 8;        // outputs per thread along the contiguous axis
static_assert(kR3 == 8, "the input-tile chunk order assumes windows that start every two chunks");
constexpr int kT1 = 4;        // output planes per CTA (and per thread)
constexpr int kMaxThreads = 256;

__host__ __device__ constexpr int ceil4(int v) { return (v + 3) & ~3; }

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool pred)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int sz = pred ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Block-wide FP64 sum; every thread passes its value, thread 0 gets the total.
__device__ __forceinline__ double block_sum_f64(double v, double* s_red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; i++) t += s_red[i];
    return t;
}

// Shared-memory layout of one CTA (in floats):
//   [input tile, 2 buffers][template ring, T1+1 planes][running totals][FP64 scratch]
// Each input-tile row stores its 16-byte chunks even chunks first, then odd
// chunks (chunk c at slot c/2, or neven + c/2 for odd c).  A thread's window
// of R3 = 8 columns starts at chunk 2*tx, so its k-th float4 load is chunk
// 2*tx + k: in this order consecutive threads read consecutive slots and the
// 128-bit loads are free of bank conflicts (in column order the 32-byte
// stride between threads puts two threads of each quarter warp on the same
// banks).
// The template ring holds plane j1 in slot j1 mod (T1+1): consecutive input
// planes u need the template planes j1 = s1 + o1 - u of the CTA's T1 output
// planes, a window that slides by one plane per u, so one new plane is staged
// per input plane.  Running totals are stored [T1*R3][threads] (thread index
// fastest: conflict-free).
struct ConvSmem {
    int rows, pitch, neven, tile_in, wplane, tile_w, tot;
    __host__ __device__ static ConvSmem make(int ntx, int nty, int q2, int q3)
    {
        ConvSmem s;
        s.rows = nty + q2 - 1;
        s.pitch = ceil4((ntx - 1) * kR3 + ceil4(kR3 + q3 - 1));
        s.neven = (s.pitch / 4 + 1) / 2;
        s.tile_in = s.rows * s.pitch;
        s.wplane = q2 * ceil4(q3);
        s.tile_w = (kT1 + 1) * s.wplane;
        s.tot = kT1 * kR3 * ntx * nty;
        return s;
    }
    __host__ __device__ size_t floats() const
    {
        size_t f = 2 * (size_t)tile_in + (size_t)tile_w + (size_t)tot;
        return (f + 1) & ~(size_t)1;                    // 8-byte align the FP64 scratch
    }
    __host__ __device__ size_t bytes() const { return floats() * sizeof(float) + 32 * sizeof(double); }
};

__device__ __forceinline__ int ring_slot(int64_t j1) { return (int)(((j1 % (kT1 + 1)) + (kT1 + 1)) % (kT1 + 1)); }

// One CTA's output tile `tile` of volume `bidx` (batched plain calls) of the launch L.
template <int Q3>
__device__ __forceinline__ void conv_fp32_body(const ConvLaunch& L, const int ntx, const int nty, const int tiles2,
                                               const int tiles3, const int tile, const int bidx, float* smem)
{
    constexpr int R3 = kR3, T1 = kT1;
    constexpr int WLP = ceil4(R3 + Q3 - 1);
    constexpr int Q3P = ceil4(Q3);

    const ConvGeom& G = L.g;
    // The block has whole warps (blockDim.x = nthr rounded up to 32); threads
    // past nthr only help stage shared memory.
    const int tid = threadIdx.x;
    const int nthr = ntx * nty;
    const bool active = tid < nthr;
    const int tx = active ? tid % ntx : 0, ty = active ? tid / ntx : 0;
    const int lane = tid & 31, wid = tid >> 5, nwarps = blockDim.x >> 5;
    const int q1 = G.q1, q2 = G.q2;
    const ConvSmem lay = ConvSmem::make(ntx, nty, q2, Q3);
    float* s_in0 = smem;
    float* s_w = smem + 2 * lay.tile_in;
    float* s_tot = s_w + lay.tile_w;
    double* s_red = reinterpret_cast<double*>(smem + lay.floats());

    int bt = tile;
    const int t3 = bt % tiles3;
    bt /= tiles3;
    const int t2 = bt % tiles2;
    const int t1 = bt / tiles2;
    const int64_t S1 = (int64_t)t1 * T1, S2 = (int64_t)t2 * nty, S3 = (int64_t)t3 * ntx * R3;
    const float* in = L.in ? L.in + bidx * L.in_bstride : nullptr;
    float* out = L.out ? L.out + bidx * L.out_bstride : nullptr;
    const int role = L.role;
    bool do_conv = true;
    int cur = 0;
    double delta = 0.0;
    float lamf = 0.f;
    bool want_a = false, want_x = false;          // Armijo slope and ||x_t||^2 partials (adjoint trial)
    bool want_sy = false;                         // <x_k - x_{k-1}, grad f(x_k) - grad f(x_{k-1})> (bb)
    if (role == ROLE_FWD_INIT || role == ROLE_FWD_TRIAL || role == ROLE_ADJ_TRIAL) {
        const IterState* st = L.ctx.st;
        if (st->done) return;                                   // uniform: the run has finished
        cur = st->cur;
        lamf = (float)st->lambda;
        want_a = role == ROLE_ADJ_TRIAL && st->sigma != 0.0;
        want_x = role == ROLE_ADJ_TRIAL && st->lambda != 0.0;
        want_sy = role == ROLE_ADJ_TRIAL && st->bb && st->need_grad && st->accepted >= 1;
        if (role == ROLE_FWD_INIT) {
            in = L.ctx.x[cur];
            out = L.ctx.r[cur];
        } else if (role == ROLE_FWD_TRIAL) {
            in = L.ctx.x[cur ^ 1];
            out = L.ctx.r[cur ^ 1];
        } else {
            in = L.ctx.r[cur];
            out = L.ctx.g;
            delta = st->delta;
            do_conv = st->need_grad != 0;
        }
    }

    if (active)
#pragma unroll
        for (int k = 0; k < T1 * R3; k++) s_tot[k * nthr + tid] = 0.f;

    const int64_t s2 = S2 + ty;
    if (do_conv) {
        const int64_t ulo = max((int64_t)0, S1 + G.o1 - q1 + 1);
        const int64_t uhi = min(G.a1 - 1, S1 + T1 - 1 + G.o1);
        const int j2lo = (int)max((int64_t)0, s2 + G.o2 - (G.a2 - 1));
        const int j2hi = active ? (int)min((int64_t)q2 - 1, s2 + G.o2) : -1;
        const int64_t v0 = S2 + G.o2 - q2 + 1;                  // input row of shared row 0
        const int64_t c0 = S3 + G.o3 - Q3 + 1;                  // input column of shared column 0

        // one warp per shared row, lanes along the row: no index division
        auto stage_in = [&](int64_t u, int buf) {
            float* dst = s_in0 + buf * lay.tile_in;
            const float* plane = in + u * G.a2 * G.a3;
            for (int r = wid; r < lay.rows; r += nwarps) {
                const int64_t v = v0 + r;
                const bool rok = (v >= 0) && (v < G.a2);
                const float* src = plane + v * G.a3;
                for (int c = lane; c < lay.pitch; c += 32) {
                    const int64_t t = c0 + c;
                    const bool ok = rok && (t >= 0) && (t < G.a3);
                    const int c4 = c >> 2;
                    const int slot = (c4 & 1) ? lay.neven + (c4 >> 1) : (c4 >> 1);
                    cp_async4(dst + r * lay.pitch + slot * 4 + (c & 3), ok ? src + t : in, ok);
                }
            }
        };
        auto stage_w = [&](int64_t j1) {                        // template plane j1 into its ring slot
            if (j1 < 0 || j1 >= q1) return;
            float* dst = s_w + ring_slot(j1) * lay.wplane;
            const float* src = L.w + j1 * q2 * Q3;
            for (int r = wid; r < q2; r += nwarps)
                for (int c = lane; c < Q3P; c += 32)
                    cp_async4(dst + r * Q3P + c, c < Q3 ? src + r * Q3 + c : L.w, c < Q3);
        };

        if (ulo <= uhi) {
            stage_in(ulo, 0);
            for (int i = 0; i < T1; i++) stage_w(S1 + i + G.o1 - ulo);
            cp_async_commit();
            for (int64_t u = ulo; u <= uhi; ++u) {
                const int buf = (int)((u - ulo) & 1);
                if (u + 1 <= uhi) {
                    stage_in(u + 1, buf ^ 1);
                    stage_w(S1 + G.o1 - (u + 1));               // the one plane that enters the window
                }
                cp_async_commit();
                cp_async_wait1();
                __syncthreads();

                bool valid[T1];
                int woff[T1];
#pragma unroll
                for (int i = 0; i < T1; i++) {
                    const int64_t j1 = S1 + i + G.o1 - u;
                    valid[i] = (j1 >= 0) && (j1 < q1) && (S1 + i < G.b1);
                    woff[i] = ring_slot(j1) * lay.wplane;
                }
                float part[T1][R3];
#pragma unroll
                for (int i = 0; i < T1; i++)
#pragma unroll
                    for (int c = 0; c < R3; c++) part[i][c] = 0.f;

                const float* sin = s_in0 + buf * lay.tile_in + tx * 4;      // chunk 2*tx: even slot tx
                const int odd = lay.neven * 4;
                for (int j2 = j2lo; j2 <= j2hi; ++j2) {
                    const float* src = sin + (ty + q2 - 1 - j2) * lay.pitch;
                    float wv[WLP];
#pragma unroll
                    for (int i = 0; i < WLP; i += 4) {
                        const int k = i >> 2;                   // chunk 2*tx + k
                        const float4 v = *reinterpret_cast<const float4*>(src + ((k & 1) ? odd : 0) + (k >> 1) * 4);
                        wv[i] = v.x; wv[i + 1] = v.y; wv[i + 2] = v.z; wv[i + 3] = v.w;
                    }
#pragma unroll
                    for (int i = 0; i < T1; i++) {
                        if (!valid[i]) continue;
                        const float* hp = s_w + woff[i] + j2 * Q3P;
#pragma unroll
                        for (int jj = 0; jj < Q3P; jj += 4) {
                            const float4 h4 = *reinterpret_cast<const float4*>(hp + jj);
                            const float hv[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
                            for (int k = 0; k < 4; k++) {
                                const int j3 = jj + k;
                                if (j3 < Q3) {
#pragma unroll
                                    for (int c = 0; c < R3; c++)
                                        part[i][c] = fmaf(hv[k], wv[c + Q3 - 1 - j3], part[i][c]);
                                }
                            }
                        }
                    }
                }
                if (active)
#pragma unroll
                    for (int i = 0; i < T1; i++)
                        if (valid[i])
#pragma unroll
                            for (int c = 0; c < R3; c++) s_tot[(i * R3 + c) * nthr + tid] += part[i][c];
                __syncthreads();
            }
        }
    }

    // Epilogue.  Per-element arithmetic in FP32 (FP64 runs at a small fraction of
    // the FP32 rate on this GPU); each thread's squares are summed in FP32 over
    // its <= 32 outputs and the block and grid sums are FP64.
    float loc = 0.f, loc_a = 0.f, loc_x = 0.f, loc_sy = 0.f;
    const bool row_ok = active && s2 < G.b2;
    const float deltaf = (float)delta;
#pragma unroll
    for (int i = 0; i < T1; i++) {
        const int64_t s1 = S1 + i;
        if (s1 >= G.b1 || !row_ok) continue;
#pragma unroll
        for (int c = 0; c < R3; c++) {
            const int64_t s3 = S3 + (int64_t)tx * R3 + c;
            if (s3 >= G.b3) continue;
            const int64_t idx = (s1 * G.b2 + s2) * G.b3 + s3;
            const float v = s_tot[(i * R3 + c) * nthr + tid];
            switch (role) {
            case ROLE_PLAIN:
                out[idx] = v;
                break;
            case ROLE_FWD_INIT:
            case ROLE_FWD_TRIAL: {
                const float rr = v - L.ctx.y[idx];
                out[idx] = rr;
                loc = fmaf(rr, rr, loc);
                break;
            }
            case ROLE_ADJ_TRIAL: {
                float gg;
                const float xo = L.ctx.x[cur][idx];
                if (do_conv) {
                    gg = v;
                    if (want_sy) {                            // before g and x_{k-1} are overwritten
                        const float s = xo - L.ctx.x[cur ^ 1][idx];
                        loc_sy = fmaf(s, fmaf(lamf, s, v - out[idx]), loc_sy);
                    }
                    out[idx] = gg;
                } else {
                    gg = L.ctx.g[idx];
                }
                const float gt = fmaf(lamf, xo, gg);          // grad f = A^T r + lambda x (lambda = 0: A^T r)
                const float xn = fmaxf(fmaf(-deltaf, gt, xo), 0.f);
                L.ctx.x[cur ^ 1][idx] = xn;
                const float d = xn - xo;
                loc = fmaf(d, d, loc);
                loc_a = fmaf(gt, d, loc_a);
                loc_x = fmaf(xn, xn, loc_x);
                break;
            }
            case ROLE_RL_RATIO: {
                const float yv = L.y[idx];
                out[idx] = v != 0.f ? yv / v : 0.f;
                break;
            }
            case ROLE_RL_UPDATE: {
                const float nv = L.ctx.aux[idx];
                float* x = L.ctx.x[0];
                x[idx] = nv != 0.f ? x[idx] * (v / nv) : 0.f;
                break;
            }
            default:
                break;
            }
        }
    }
    if (role == ROLE_FWD_INIT || role == ROLE_FWD_TRIAL || role == ROLE_ADJ_TRIAL) {
        const double t = block_sum_f64((double)loc, s_red);
        if (tid == 0) {
            double* part = (role == ROLE_ADJ_TRIAL) ? L.ctx.part_m : L.ctx.part_f;
            part[tile] = t;
        }
        if (want_a) {                                           // uniform
            __syncthreads();                                    // s_red is reused
            const double ta = block_sum_f64((double)loc_a, s_red);
            if (tid == 0) L.ctx.part_a[tile] = ta;
        }
        if (want_x) {
            __syncthreads();
            const double tx2 = block_sum_f64((double)loc_x, s_red);
            if (tid == 0) L.ctx.part_x[tile] = tx2;
        }
        if (want_sy) {
            __syncthreads();
            const double tsy = block_sum_f64((double)loc_sy, s_red);
            if (tid == 0) L.ctx.part_sy[tile] = tsy;
        }
    }
}

template <int Q3>
__global__ void __launch_bounds__(kMaxThreads, 2)
conv_fp32_kernel(const ConvLaunch L, const int ntx, const int nty, const int tiles2, const int tiles3)
{
    extern __shared__ __align__(16) float smem[];
    conv_fp32_body<Q3>(L, ntx, nty, tiles2, tiles3, blockIdx.x, blockIdx.y, smem);
}

// Batched form: CTA i computes tile items[i].y of volume items[i].x, each volume with its own
// geometry, buffers and tile shape (all volumes of one launch share the template width Q3).
template <int Q3>
__global__ void __launch_bounds__(kMaxThreads, 2) conv_fp32_batch_kernel(const ConvBatchVol* vols, const int2* items)
{
    extern __shared__ __align__(16) float smem[];
    const int2 it = items[blockIdx.x];
    const ConvBatchVol& V = vols[it.x];
    conv_fp32_body<Q3>(V.L, V.ntx, V.nty, V.tiles2, V.tiles3, it.y, 0, smem);
}

template <int Q3>
cudaError_t conv_fp32_batch_launch_q(const ConvBatchVol* vols, const int2* items, int nitems, size_t smem, cudaStream_t s)
{
    if (nitems <= 0)
        return cudaFuncSetAttribute(conv_fp32_batch_kernel<Q3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    conv_fp32_batch_kernel<Q3><<<nitems, kMaxThreads, smem, s>>>(vols, items);
    return cudaGetLastError();
}

template <int Q3>
cudaError_t conv_fp32_launch_q(const ConvLaunch& L, const ConvTile& t, cudaStream_t s)
{
    if (L.batch == 0) {       // preparation call (outside any stream capture): opt in to large shared memory
        return cudaFuncSetAttribute(conv_fp32_kernel<Q3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    }
    dim3 grid((unsigned)t.grid, (unsigned)L.batch);
    const int threads = (t.ntx * t.nty + 31) & ~31;
    conv_fp32_kernel<Q3><<<grid, threads, t.smem, s>>>(L, t.ntx, t.nty, t.tiles2, t.tiles3);
    return cudaGetLastError();
}

#define CDV_INSTANTIATE_FP32(Q)                                                                       \
    template cudaError_t conv_fp32_launch_q<Q>(const ConvLaunch&, const ConvTile&, cudaStream_t);       \
    template cudaError_t conv_fp32_batch_launch_q<Q>(const ConvBatchVol*, const int2*, int, size_t, cudaStream_t);
#define CDV_EXTERN_FP32(Q)                                                                            \
    extern template cudaError_t conv_fp32_launch_q<Q>(const ConvLaunch&, const ConvTile&, cudaStream_t); \
    extern template cudaError_t conv_fp32_batch_launch_q<Q>(const ConvBatchVol*, const int2*, int, size_t, cudaStream_t);

}  // namespace cdv

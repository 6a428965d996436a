// Persistent batched solver: the whole K-step run of every volume of a batch in one launch.
//
// Each volume steps through phases: 0 the initial forward (r_0 = A x_0 - y), then alternately an
// adjoint trial (odd phases: g = A^T r_k and the projected update x_t) and a forward trial (even
// phases >= 2: r_t = A x_t - y), Steps 1-3 of the iteration.  A phase is the volume's FP32-engine
// tiles of that direction; the CTAs of the launch take tiles from any volume whose current phase has
// tiles left, through one 64-bit word per volume (phase in the high half, next tile in the low half,
// taken with atomicAdd, so a tile index always comes with the phase it belongs to; warp 0 of a CTA
// scans 32 of these words per load).  The CTA that completes a phase's last tile runs that volume's
// step rule (after a forward: the FP64 decision of Step 2, in the fixed order of the 512-thread
// decision kernel) and opens the next phase, or retires the volume.  No CTA waits for another CTA's
// result: a CTA without a tile to take scans again after a short sleep, so the launch needs no
// co-residency and cannot deadlock; a CTA that finds no tile for the batch plan's idle budget
// (cdv_batch_set_wait_cycles) records CDV_ERR_TIMEOUT, and every CTA leaves at its next look.  Every
// tile writes its FP64 partials at its own index, and the decisions sum them in the same order as the
// per-slot launches, so each volume's iterates equal those of the per-slot batched solver and of
// cdv_iterate on it alone.
#include <algorithm>

#include "conv_fp32.cuh"
#include "decide.cuh"

namespace cdv {

namespace {

constexpr unsigned kPhaseDone = 0xFFFFFFFFu;

// One tile, in a function of its own per template width (compiled and register-allocated apart from
// the scheduling loop and from the other widths)
template <int Q3>
__device__ __noinline__ void persist_tile_q(const ConvBatchVol& V, int tile, float* smem)
{
    conv_fp32_body<Q3>(V.L, V.ntx, V.nty, V.tiles2, V.tiles3, tile, 0, smem);
}

__device__ void persist_tile(const ConvBatchVol& V, int tile, float* smem)
{
    switch (V.L.g.q3) {
#define CDV_CASE(Q) \
    case Q: persist_tile_q<Q>(V, tile, smem); break;
        CDV_CASE(1) CDV_CASE(3) CDV_CASE(5) CDV_CASE(7) CDV_CASE(9) CDV_CASE(11) CDV_CASE(13) CDV_CASE(15)
        CDV_CASE(17) CDV_CASE(19) CDV_CASE(21) CDV_CASE(23) CDV_CASE(25) CDV_CASE(27) CDV_CASE(29) CDV_CASE(31)
#undef CDV_CASE
    default:
        break;
    }
}

// tiles of a phase: the adjoint's (odd phases, y) or the forward's (x)
__device__ __forceinline__ int phase_tiles(int2 nt, unsigned ph) { return (ph & 1u) ? nt.y : nt.x; }

}  // namespace

__global__ void __launch_bounds__(kMaxThreads, 2) conv_fp32_persist_kernel(const BatchPersist P)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_kind, s_pos, s_tile, s_last;
    __shared__ unsigned s_phase;
    const int tid = threadIdx.x;
    bool idle = false;                              // thread 0: since when no tile was found
    long long idle0 = 0;
    for (;;) {
        if (tid < 32) {
            // warp 0 scans 32 volumes per step (their words and tile counts are stored in scan order) and
            // tries the ones with tiles left, lowest position first.
            // kind: 0 initial forward, 1 adjoint trial, 2 forward trial, -1 nothing to take, -2 leave
            int kind = -1;
            if (*(volatile int*)P.vols_done >= P.count || *(volatile int*)P.err != 0) kind = -2;
            for (int base = 0; kind == -1 && base < P.count; base += 32) {
                const int k = base + tid;
                bool avail = false;
                if (k < P.count) {
                    const unsigned long long w = *(volatile unsigned long long*)&P.word[k];
                    const unsigned ph = (unsigned)(w >> 32);
                    avail = ph != kPhaseDone && (unsigned)w < (unsigned)phase_tiles(P.ntiles[k], ph);
                }
                unsigned mask = __ballot_sync(0xffffffffu, avail);
                while (mask && kind == -1) {
                    const int lead = __ffs(mask) - 1;
                    unsigned long long o = 0;
                    if (tid == lead) o = atomicAdd(&P.word[base + lead], 1ull);
                    o = __shfl_sync(0xffffffffu, o, lead);
                    const unsigned ph2 = (unsigned)(o >> 32);
                    if (ph2 != kPhaseDone && (unsigned)o < (unsigned)phase_tiles(P.ntiles[base + lead], ph2)) {
                        kind = ph2 == 0 ? 0 : ((ph2 & 1u) ? 1 : 2);
                        if (tid == 0) {
                            s_pos = base + lead;
                            s_tile = (int)(unsigned)o;
                            s_phase = ph2;
                        }
                    }
                    mask &= mask - 1;
                }
            }
            if (tid == 0) {
                if (kind == -1) {
                    if (!idle) {
                        idle = true;
                        idle0 = clock64();
                    } else if (clock64() - idle0 > P.wait_cycles) {
                        atomicExch(P.err, (int)CDV_ERR_TIMEOUT);
                        kind = -2;
                    }
                } else {
                    idle = false;
                }
                s_kind = kind;
                __threadfence();                    // acquire: the phase's inputs and state are visible
            }
        }
        __syncthreads();
        const int kind = s_kind;
        if (kind == -2) break;
        if (kind == -1) {
            __nanosleep(400);
            __syncthreads();                        // everyone has read s_kind before thread 0 writes it
            continue;
        }
        const int pos = s_pos, tile = s_tile, v = P.order[pos];
        const unsigned ph = s_phase;
        const ConvBatchVol& V = kind == 0 ? P.fi[v] : (kind == 1 ? P.at[v] : P.ft[v]);
        persist_tile(V, tile, smem);
        __syncthreads();
        if (tid == 0) {
            __threadfence();                        // release this tile's outputs and partials
            s_last = atomicAdd(&P.tiles_done[v], 1) == phase_tiles(P.ntiles[pos], ph) - 1;
            if (s_last) __threadfence();            // acquire every other tile of the phase
        }
        __syncthreads();
        if (s_last) {
            const BatchVolCtx& b = P.ctx[v];
            unsigned next = ph + 1;
            if (kind != 1) {
                double* sh = reinterpret_cast<double*>(smem);     // the tile's shared memory is free now
                decide_body_r(b.c, b.nparts_f, b.nparts_m, kind == 0 ? 1 : 0, sh, Reduce512On256{});
            }
            if (tid == 0) {
                if (kind != 1) {
                    const IterState* st = b.c.st;
                    if (st->done || st->trials >= P.max_trials) next = kPhaseDone;
                }
                P.tiles_done[v] = 0;
                __threadfence();                    // release the state before the next phase opens
                atomicExch(&P.word[pos], (unsigned long long)next << 32);
                if (next == kPhaseDone) atomicAdd(P.vols_done, 1);
            }
        }
        __syncthreads();
    }
}

cudaError_t conv_fp32_persist_prepare()
{
    // tiles take at most 110 KB (two CTAs per SM); the kernel also has a few static words
    return cudaFuncSetAttribute(conv_fp32_persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

int conv_fp32_persist_grid(size_t smem)
{
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, conv_fp32_persist_kernel, kMaxThreads, smem) != cudaSuccess)
        return 0;
    return nsm * std::max(per, 1);
}

cudaError_t conv_fp32_persist_launch(const BatchPersist& P, int grid, size_t smem, cudaStream_t s)
{
    if (grid < 1 || P.count < 1) return cudaErrorInvalidValue;
    conv_fp32_persist_kernel<<<grid, kMaxThreads, smem, s>>>(P);
    return cudaGetLastError();
}

}  // namespace cdv

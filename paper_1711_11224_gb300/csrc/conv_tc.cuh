// Tensor-core (tcgen05) direct convolution: implicit GEMM with a Toeplitz
// operand along the contiguous axis.
//
// For the generic operator out[s] = sum_j w[j] in[s + o - j] (forward:
// in = X, o = 0, w = H; adjoint: in = R, o = 2p, w = H~), fix the template
// plane j1 and row j2.  The sum over j3 for W (8 or 16) consecutive output
// columns is an input window of K >= W + q3 - 1 columns times a banded
// Toeplitz matrix T_{j1,j2}[k, n] = w[j1, j2, n + D - k].  With 128
// consecutive output rows as M this is one tcgen05.mma per 16-wide K step:
//     D_{s1}[row, n] += A_{u, j2}[row, k] * T_{s1+o1-u, j2}[k, n]
// where A_{u, j2} is input plane u read at rows shifted by j2.
//
// Shapes chosen for the tensor pipe and for the supply of template tiles:
//  * N = W x (output planes): one input plane u and template row j2 feed the
//    CTA's P = 128 / W output planes through Toeplitz tiles of consecutive
//    j1, stored side by side in 8-row groups ([j2][j1, n/8][K chunk][n%8]),
//    so one MMA with N <= 128 updates all of them and one bulk copy per
//    precision part fetches a stage.  The tensor pipe executes K / q3 times the
//    algorithmic work; the host picks W per direction from a cycle model
//    (W = 8 halves K for templates about 20 wide: K = 32 instead of 48).
//  * Two M tiles of 128 rows per CTA: every template-tile stage feeds both,
//    which halves the template bytes streamed from L2 per MMA; the stages
//    were the limiter with one M tile.  Split-BF16x3 issues hi*hi and hi*lo
//    back to back with the A operand kept in the tensor core's collector
//    buffer, so A is read from shared memory twice per three products.
//  * The row shift j2 is a 16-byte shift of the shared-memory descriptor of
//    one TMA-staged tile of plane u (K-major, no swizzle: core matrices of
//    8 rows x 16 bytes, rows 16 bytes apart), so the tile serves all q2 rows.
//  * Two-level accumulation: the contribution of each input plane goes to a
//    fresh TMEM partial (two buffers x two M tiles x 128 columns = all 512
//    columns), which epilogue warps add into FP32 register totals while the
//    MMAs of the next plane run.  One TMEM accumulator over all q1*q2
//    template rows drifts (the tensor core's FP32 accumulation truncates):
//    1e-4 relative for a 31x31x21 template.
//  * Persistent CTAs, one per SM, walk the output tiles with their ring and
//    accumulator counters carried across tiles, so a tile's stores overlap
//    the next tile's loads and MMAs.
//
// Warp roles (320 threads):
//   warp 0      TMA producer: per input plane, the A tile (per 16-byte K chunk
//               two boxes of rows/2 rows, zero-filled outside the volume) and,
//               per template row, the Toeplitz tiles of the planes in range
//               (bulk copies through a ring of stages).
//   warp 1      MMA issuer: the whole warp runs the loop with warp-uniform
//               descriptors and one elected lane issues each MMA (three for
//               split-BF16x3); tcgen05.commit releases ring stages and hands
//               each plane's partial to the epilogue.  A single thread
//               computing its own descriptors issued an MMA only every ~90
//               cycles, slower than the tensor pipe at N = 128.
//   warps 2-9   epilogue, one output row per thread, warpgroup g owning M
//               tile g: drains the partials, then the fused epilogue of the
//               FP32 engine plus the BF16/TF32 shadows the next convolution
//               reads, stored through a per-warp staging tile so that warp
//               accesses cover rows of 8 consecutive columns.
// Every wait is bounded (the plan's budget, about 0.5 s by default).  A wait that runs out records
// CDV_ERR_TIMEOUT in the device error word; the CTA stops issuing work, waits
// for its own copies and MMAs, frees its TMEM and exits.  CTAs that start
// after an error has been recorded skip their work.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "cdv_internal.h"

namespace cdv {

namespace {

constexpr int kM = 128;
constexpr int kNT = 128;       // accumulator columns per M tile: W output columns x P = 128 / W planes
constexpr int kMT = 2;         // 128-row M tiles per CTA: each template-tile stage feeds both
constexpr int kEC = 8;         // columns per staged store block
constexpr int kThreads = 320;

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(unsigned addr, unsigned lbo, unsigned sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait for the phase of the given parity; false after `budget` cycles (the work loops use the
// plan's budget, 1e9 cycles or about 0.5 s by default; the drain before exit always kDrainCycles).
constexpr long long kDrainCycles = 2000000000ll;
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Non-blocking probe of the phase (try_wait may suspend the thread until the phase completes).
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Budgets below this are probed without suspending, so the clock alone decides when they run out.
constexpr long long kPollBelow = 1000000ll;
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long budget = kDrainCycles)
{
    const bool poll = budget < kPollBelow;
    if (poll ? mbar_test(bar, parity) : mbar_try(bar, parity)) return true;   // fast path: no clock reads
    const long long t0 = clock64();
    for (;;) {
        if (poll ? mbar_test(bar, parity) : mbar_try(bar, parity)) return true;
        if (clock64() - t0 > budget) return false;
    }
}
__device__ __forceinline__ void tma3(unsigned dst, const CUtensorMap* map, int x, int y, int z, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// One K step of the product on the tensor core, issued by one elected lane of a converged warp
// (the operands are warp-uniform).  Split-BF16x3: hi*hi and hi*lo share A, the second reusing it
// from the collector buffer, then lo*hi.
template <int KIND>
__device__ __forceinline__ void mma_step(unsigned d, uint64_t ah, uint64_t al, uint64_t bh, uint64_t bl, unsigned idesc,
                                         unsigned acc)
{
    if (KIND == CDV_MODE_SPLIT_BF16X3)
        asm volatile(
            "{\n .reg .pred p, q, e;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %6, 0;\n setp.ne.b32 q, 1, 0;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %3, %5, p;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %4, %5, q;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %3, %5, q;\n}\n" ::"r"(d),
            "l"(ah), "l"(al), "l"(bh), "l"(bl), "r"(idesc), "r"(acc));
    else if (KIND == CDV_MODE_TF32)
        asm volatile(
            "{\n .reg .pred p, e;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
            " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(ah), "l"(bh), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n .reg .pred p, e;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(ah), "l"(bh), "r"(idesc), "r"(acc));
}
// tcgen05.commit from the elected lane (the one that issued the MMAs)
__device__ __forceinline__ void mma_commit_elect(unsigned bar)
{
    asm volatile(
        "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(bar)
        : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
template <int W>
__device__ __forceinline__ void tmem_ld(unsigned taddr, float* v);
template <>
__device__ __forceinline__ void tmem_ld<8>(unsigned taddr, float* v)
{
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}
template <>
__device__ __forceinline__ void tmem_ld<16>(unsigned taddr, float* v)
{
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// Shadow value(s) of an FP32 result for the next tensor-core convolution.
template <int KIND>
__device__ __forceinline__ void store_shadow(void* hi, void* lo, int64_t i, float v)
{
    if (KIND == CDV_MODE_TF32) {
        unsigned t;
        asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(t) : "f"(v));
        reinterpret_cast<unsigned*>(hi)[i] = t;
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        reinterpret_cast<__nv_bfloat16*>(hi)[i] = h;
        if (KIND == CDV_MODE_SPLIT_BF16X3)
            reinterpret_cast<__nv_bfloat16*>(lo)[i] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

}  // namespace

// Shared-memory layout of one CTA (bytes).
struct TcSmem {
    size_t a_bytes, b_bytes, off_b, off_bar, off_stage, total;
    __host__ __device__ static TcSmem make(const TcArgs& t)
    {
        TcSmem s;
        s.a_bytes = (size_t)t.kchunks * t.rows * 16;              // one part of one input plane
        s.b_bytes = (size_t)t.kchunks * t.P * t.W * 16;          // one part of one ring stage
        s.off_b = (size_t)t.na * t.nprec * s.a_bytes;
        s.off_bar = s.off_b + (size_t)t.ns * t.nprec * s.b_bytes;
        s.off_stage = s.off_bar + 512;
        s.total = s.off_stage + (size_t)(kThreads / 32 - 2) * 32 * kEC * 4;   // 32 x 8 floats per epilogue warp
        return s;
    }
};


// One output tile: planes [S1, S1 + P), rows [S2, S2 + 256), columns [S3, S3 + W), and the input
// planes [ulo, uhi] that reach it.
struct TcTile {
    int64_t S1, S2, S3, s1_end, ulo, uhi;
    __device__ static TcTile make(const TcArgs& T, int tile)
    {
        TcTile c;
        const int t3 = tile % T.tiles3;
        tile /= T.tiles3;
        const int t2 = tile % T.tiles2;
        const int t1 = tile / T.tiles2;
        const ConvGeom& G = T.g;
        c.S1 = (int64_t)t1 * T.P;
        c.S2 = (int64_t)t2 * kM * kMT;
        c.S3 = (int64_t)t3 * T.W;
        c.s1_end = min(c.S1 + T.P, G.b1);
        c.ulo = max((int64_t)0, c.S1 + G.o1 - G.q1 + 1);
        c.uhi = min(G.a1 - 1, c.s1_end - 1 + G.o1);
        return c;
    }
    // output planes of the tile that input plane u reaches: [ilo, ihi] (relative to S1)
    __device__ void plane_range(const ConvGeom& G, int64_t u, int& ilo, int& ihi) const
    {
        ilo = (int)max((int64_t)0, u - G.o1 - S1);
        ihi = (int)min(s1_end - 1 - S1, u - G.o1 + G.q1 - 1 - S1);
    }
    // Planes [lo, hi] the MMA covers for planes [ilo, ihi] in range: N = W x planes must be a multiple
    // of 16, so with W = 8 an odd count takes one neighbouring plane of the tile (its accumulator
    // columns are never drained; whatever its template slot holds reaches only those columns, since
    // column n of the product reads only column n of B).  Returns the padded planes in front (0 or 1).
    template <int W, int P>
    __device__ static int padded(int ilo, int ihi, int& lo, int& hi)
    {
        lo = ilo;
        hi = ihi;
        if (W == 8 && ((ihi - ilo + 1) & 1)) {
            if (ihi < P - 1) hi = ihi + 1;
            else { lo = ilo - 1; return 1; }
        }
        return 0;
    }
};

// VAR: the step-rule variants of the iteration (Tikhonov term, Armijo slope, Barzilai-Borwein inner
// product) in the adjoint epilogue; a separate instantiation, so the default kernel keeps its registers.
template <int KIND, int W, bool VAR>
__global__ void __launch_bounds__(kThreads, 1)
conv_tc_kernel(const __grid_constant__ TcArgs T, const __grid_constant__ CUtensorMap mh0,
               const __grid_constant__ CUtensorMap ml0, const __grid_constant__ CUtensorMap mh1,
               const __grid_constant__ CUtensorMap ml1)
{
    constexpr int NPREC = (KIND == CDV_MODE_SPLIT_BF16X3) ? 2 : 1;
    constexpr int EPT = (KIND == CDV_MODE_TF32) ? 4 : 8;       // elements per 16-byte K chunk
    constexpr int P = kNT / W;                                 // output planes per CTA
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const TcSmem lay = TcSmem::make(T);
    const ConvGeom& G = T.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int role = T.role;
    int sel = 0, cur = 0;
    bool do_conv = true;
    float delta = 0.f, lamf = 0.f;
    bool want_a = false, want_x = false;      // Armijo slope and ||x_t||^2 partials (adjoint trial)
    bool want_sy = false;                     // <x_k - x_{k-1}, grad f(x_k) - grad f(x_{k-1})> (bb)
    float* out = T.out;
    const float* xin = nullptr;
    if (role == ROLE_FWD_INIT || role == ROLE_FWD_TRIAL || role == ROLE_ADJ_TRIAL) {
        const IterState* st = T.ctx.st;
        if (st->done) return;
        cur = st->cur;
        if (VAR) {
            lamf = (float)st->lambda;
            want_a = role == ROLE_ADJ_TRIAL && st->sigma != 0.0;
            want_x = role == ROLE_ADJ_TRIAL && st->lambda != 0.0;
            want_sy = role == ROLE_ADJ_TRIAL && st->bb && st->need_grad && st->accepted >= 1;
        }
        if (role == ROLE_FWD_INIT) {
            sel = cur;
            out = T.ctx.r[cur];
        } else if (role == ROLE_FWD_TRIAL) {
            sel = cur ^ 1;
            out = T.ctx.r[cur ^ 1];
        } else {
            sel = cur;
            out = T.ctx.g;
            xin = T.ctx.x[cur];
            delta = (float)st->delta;
            do_conv = st->need_grad != 0;
        }
    }
    const CUtensorMap* map_hi = sel ? &mh1 : &mh0;
    const CUtensorMap* map_lo = sel ? &ml1 : &ml0;

    unsigned char* sA = sm;
    unsigned char* sB = sm + lay.off_b;
    // barriers: a_full[2] a_empty[2] b_full[16] b_empty[16] acc_full[2] acc_free[2] drain
    const unsigned bar0 = su32(sm + lay.off_bar);
    auto A_FULL = [&](int i) { return bar0 + 8u * i; };
    auto A_EMPTY = [&](int i) { return bar0 + 8u * (2 + i); };
    auto B_FULL = [&](int i) { return bar0 + 8u * (4 + i); };
    auto B_EMPTY = [&](int i) { return bar0 + 8u * (20 + i); };
    auto ACC_FULL = [&](int i) { return bar0 + 8u * (36 + i); };
    auto ACC_FREE = [&](int i) { return bar0 + 8u * (38 + i); };
    const unsigned DRAIN = bar0 + 8u * 40;
    unsigned* tslot = reinterpret_cast<unsigned*>(sm + lay.off_bar + 384);
    volatile int* sflag = reinterpret_cast<volatile int*>(sm + lay.off_bar + 392);

    // Persistent CTAs: tiles blockIdx.x, blockIdx.x + gridDim.x, ...  Every role walks the same
    // sequence and keeps its ring and accumulator counters across tiles, so the epilogue of one
    // tile overlaps the loads and MMAs of the next.
    const int ntiles = T.ntiles;
    const bool run = do_conv && *(volatile int*)T.err == 0;

    if (tid == 0) {
        for (int i = 0; i < 38; i++) mbar_init(bar0 + 8u * i, 1);
        mbar_init(ACC_FREE(0), 8);
        mbar_init(ACC_FREE(1), 8);
        mbar_init(DRAIN, 1);
        *sflag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    const unsigned tcols = T.tmem_cols;
    if (run && warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tslot)), "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = run ? *tslot : 0u;

    const int half = T.rows / 2;
    const int ksteps = T.K / (2 * EPT);
    auto fail = [&]() {
        *sflag = 1;
        atomicExch(T.err, (int)CDV_ERR_TIMEOUT);
    };

    if (run && warp == 0 && lane == 0) {
        // ---------------- TMA producer
        int bs = 0, it = 0, nb = 0;
        unsigned bph = 0;
        int a_uses[2] = {0, 0};
        for (int tile = blockIdx.x; tile < ntiles && !*sflag; tile += gridDim.x) {
            const TcTile C = TcTile::make(T, tile);
            const int64_t ws = C.S3 + G.o3 - (G.q3 - 1) - T.e;      // input column of K index 0
            const int64_t v0 = C.S2 + G.o2 - (G.q2 - 1);            // input row of staged row 0
            for (int64_t u = C.ulo; u <= C.uhi && !*sflag; ++u, ++it) {
                const int ab = it % T.na;
                if (!mbar_wait(A_EMPTY(ab), (unsigned)(((it / T.na) & 1) ^ 1), T.wait_cycles)) { fail(); break; }
                mbar_expect_tx(A_FULL(ab), (unsigned)(NPREC * lay.a_bytes));
                a_uses[ab] = it / T.na + 1;
                for (int p = 0; p < NPREC; p++) {
                    const CUtensorMap* mp = p ? map_lo : map_hi;
                    const unsigned dst = su32(sA + ((size_t)ab * NPREC + p) * lay.a_bytes);
                    for (int c = 0; c < T.kchunks; c++)
                        for (int h = 0; h < 2; h++)
                            tma3(dst + (unsigned)((c * T.rows + h * half) * 16), mp, (int)(ws + c * EPT),
                                 (int)(v0 + h * half), (int)u, A_FULL(ab));
                }
                int ilo, ihi, lo, hi;
                C.plane_range(G, u, ilo, ihi);
                const int front = TcTile::padded<W, P>(ilo, ihi, lo, hi);
                const int64_t j1lo = C.S1 + ilo + G.o1 - u;
                const int nv = ihi - ilo + 1;
                for (int j2 = 0; j2 < G.q2; j2++) {
                    if (!mbar_wait(B_EMPTY(bs), bph ^ 1, T.wait_cycles)) { fail(); break; }
                    mbar_expect_tx(B_FULL(bs), (unsigned)(NPREC * T.kchunks * nv * W * 16));
                    for (int p = 0; p < NPREC; p++) {
                        const unsigned char* src0 = reinterpret_cast<const unsigned char*>(T.bt[p]);
                        // the tiles of planes j1lo .. j1lo + nv - 1 of template row j2 are one contiguous run
                        const unsigned dst =
                            su32(sB + ((size_t)bs * NPREC + p) * lay.b_bytes) + (unsigned)(front * W * T.kchunks * 16);
                        const size_t grp = ((size_t)j2 * G.q1 + (size_t)j1lo) * (W / 8);
                        bulk_g2s(dst, src0 + grp * T.kchunks * 128, (unsigned)(nv * W * T.kchunks * 16), B_FULL(bs));
                    }
                    ++nb;
                    if (++bs == T.ns) { bs = 0; bph ^= 1; }
                }
            }
        }
        // make sure every copy this thread issued has landed before the CTA may exit
        for (int ab = 0; ab < T.na; ab++)
            if (a_uses[ab] > 0) mbar_wait(A_FULL(ab), (unsigned)((a_uses[ab] - 1) & 1));
        for (int k = 0; k < T.ns && k < nb; k++) {
            const int idx = nb - 1 - k;                           // the last use of each stage
            mbar_wait(B_FULL(idx % T.ns), (unsigned)((idx / T.ns) & 1));
        }
    } else if (run && warp == 1) {
        // ---------------- MMA issuer: the whole warp runs the loop (all values warp-uniform) and one
        // elected lane issues each MMA and commit.  Descriptors are templates with a zero start
        // address plus the start in 16-byte units, which cannot carry out of the 14-bit field for
        // CTA-local offsets below 256 KB.
        const unsigned fmt = (KIND == CDV_MODE_TF32) ? 2u : 1u;
        // A: [K chunk][row][16 B] (K neighbours rows x 16 B apart, 8-row groups 128 B apart);
        // B: [8-row group][K chunk][8 rows][16 B] (K neighbours 128 B apart, groups kchunks x 128 B)
        const unsigned lbo_a = (unsigned)T.rows * 16;
        const uint64_t da0 = sdesc(0, lbo_a, 128), db0 = sdesc(0, 128, (unsigned)T.kchunks * 128);
        const uint64_t a_kstep = (2u * lbo_a) >> 4, b_kstep = (2u * 128u) >> 4;
        // CTA-local offsets only (as sdesc masks): in a cluster launch the shared-window address also
        // carries the CTA's rank above bit 18, which must not reach the descriptor
        const unsigned sA16 = (su32(sA) & 0x3FFFFu) >> 4, sB16 = (su32(sB) & 0x3FFFFu) >> 4;
        const unsigned a_part16 = (unsigned)(lay.a_bytes >> 4), b_part16 = (unsigned)(lay.b_bytes >> 4);
        int bs = 0, it = 0;
        unsigned bph = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const TcTile C = TcTile::make(T, tile);
            const int nmt = (int)min((int64_t)kMT, (G.b2 - C.S2 + kM - 1) / kM);   // M tiles holding output rows
            for (int64_t u = C.ulo; u <= C.uhi; ++u, ++it) {
                const int b = it & 1;
                const int ab = it % T.na;
                bool w = it < 2 || mbar_wait(ACC_FREE(b), (unsigned)(((it >> 1) - 1) & 1), T.wait_cycles);
                w = w && mbar_wait(A_FULL(ab), (unsigned)((it / T.na) & 1), T.wait_cycles);
                if (!__all_sync(0xffffffffu, w && !*sflag)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                int ilo, ihi, lo, hi;
                C.plane_range(G, u, ilo, ihi);
                TcTile::padded<W, P>(ilo, ihi, lo, hi);
                const unsigned n = (unsigned)(W * (hi - lo + 1));
                const unsigned idesc =
                    (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((unsigned)(kM >> 4) << 24);
                const unsigned d = tmem + (unsigned)(b * kNT + lo * W);
                // A of this plane, first row of the shift for j2 = 0 (q2 - 1 rows down)
                const unsigned a_hi = sA16 + (unsigned)(ab * NPREC) * a_part16 + (unsigned)(G.q2 - 1);
                const unsigned a_lo = a_hi + (unsigned)(NPREC - 1) * a_part16;
                unsigned acc = 0;                                          // fresh partial per input plane
                for (int j2 = 0; j2 < G.q2; j2++) {
                    if (!__all_sync(0xffffffffu, mbar_wait(B_FULL(bs), bph, T.wait_cycles))) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const unsigned b_hi = sB16 + (unsigned)(bs * NPREC) * b_part16;
                    const uint64_t bh = db0 + b_hi, bl = db0 + b_hi + (unsigned)(NPREC - 1) * b_part16;
                    const uint64_t ah = da0 + (a_hi - (unsigned)j2), al = da0 + (a_lo - (unsigned)j2);
#pragma unroll 4
                    for (int k = 0; k < ksteps; k++) {
                        const uint64_t ka = (uint64_t)k * a_kstep, kb = (uint64_t)k * b_kstep;
#pragma unroll
                        for (int mt = 0; mt < kMT; mt++) {
                            if (mt >= nmt) break;
                            // M tile mt: rows 128 mt.. of the staged plane, its own partial columns
                            const uint64_t am = ka + (uint64_t)(mt * kM);
                            mma_step<KIND>(d + (unsigned)(mt * 2 * kNT), ah + am, al + am, bh + kb, bl + kb, idesc, acc);
                        }
                        acc = 1u;
                    }
                    mma_commit_elect(B_EMPTY(bs));
                    if (++bs == T.ns) { bs = 0; bph ^= 1; }
                }
                if (!ok) break;
                mma_commit_elect(A_EMPTY(ab));
                mma_commit_elect(ACC_FULL(b));
            }
        }
        if (!ok && lane == 0) fail();
        mma_commit_elect(DRAIN);                                  // completes when every issued MMA has
        if (!__all_sync(0xffffffffu, mbar_wait(DRAIN, 0)) && lane == 0) fail();
    }

    // ---------------- epilogue (warps 2..9): one output row per thread; warpgroup g drains and owns
    // M tile g (TMEM lanes are reached by warp index mod 4, so each warpgroup covers all 128 rows)
    float loc = 0.f, loc_a = 0.f, loc_x = 0.f, loc_sy = 0.f;
    if (warp >= 2) {
        const int mt = (warp - 2) >> 2;
        const int quarter = warp & 3;
        float* stg = reinterpret_cast<float*>(sm + lay.off_stage) + (warp - 2) * 32 * kEC;
        float4* stg4 = reinterpret_cast<float4*>(stg);
        bool ok = true;
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const TcTile C = TcTile::make(T, tile);
            const bool rows_in = C.S2 + mt * kM < G.b2;               // warp-uniform: M tile holds outputs
            float tot[P][W];
#pragma unroll
            for (int i = 0; i < P; i++)
#pragma unroll
                for (int c = 0; c < W; c++) tot[i][c] = 0.f;
            if (run) {
                for (int64_t u = C.ulo; u <= C.uhi; ++u, ++it) {
                    const int b = it & 1;
                    bool w = mbar_wait(ACC_FULL(b), (unsigned)((it >> 1) & 1), T.wait_cycles);
                    w = __all_sync(0xffffffffu, w && !*sflag);
                    if (!w) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    int ilo, ihi;
                    C.plane_range(G, u, ilo, ihi);
                    if (rows_in) {
#pragma unroll
                        for (int i = 0; i < P; i++) {
                            if (i < ilo || i > ihi) continue;             // warp-uniform
                            float v[W];
                            tmem_ld<W>(tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)((mt * 2 + b) * kNT + i * W), v);
#pragma unroll
                            for (int c = 0; c < W; c++) tot[i][c] += v[c];
                        }
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(ACC_FREE(b));
                }
            }
            if (!ok) break;
            // Stores go through a per-warp 32 x 8 staging tile so that each warp instruction touches
            // four output rows of 8 consecutive columns instead of 32 rows of one column.  Row r's two
            // 16-byte halves swap places when bit 2 of r is set: conflict-free on both sides.
            if (!rows_in) continue;
#pragma unroll
            for (int q = 0; q < P * (W / kEC); q++) {
                const int i = q / (W / kEC), h = q % (W / kEC);           // plane, 8-column block
                const int64_t s1 = C.S1 + i;
                if (s1 >= G.b1) continue;                                 // warp-uniform
                __syncwarp();
                const int sw = (lane >> 2) & 1;
                stg4[lane * 2 + sw] = make_float4(tot[i][8 * h + 0], tot[i][8 * h + 1], tot[i][8 * h + 2], tot[i][8 * h + 3]);
                stg4[lane * 2 + (sw ^ 1)] =
                    make_float4(tot[i][8 * h + 4], tot[i][8 * h + 5], tot[i][8 * h + 6], tot[i][8 * h + 7]);
                __syncwarp();
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const int r = k * 4 + (lane >> 3), c = lane & 7;
                    const float v = stg[r * 8 + ((((c >> 2) ^ (k & 1))) << 2) + (c & 3)];
                    const int64_t s2 = C.S2 + mt * kM + quarter * 32 + r;
                    const int64_t s3 = C.S3 + h * kEC + c;
                    if (s2 >= G.b2 || s3 >= G.b3) continue;
                    const int64_t idx = (s1 * G.b2 + s2) * G.b3 + s3;
                    const int64_t sidx = (s1 * G.b2 + s2) * T.sh_pitch + s3;
                    switch (role) {
                    case ROLE_PLAIN:
                        out[idx] = v;
                        break;
                    case ROLE_FWD_INIT:
                    case ROLE_FWD_TRIAL: {
                        const float rr = v - T.ctx.y[idx];
                        out[idx] = rr;
                        store_shadow<KIND>(T.sh_out_hi[sel], T.sh_out_lo[sel], sidx, rr);
                        loc = fmaf(rr, rr, loc);
                        break;
                    }
                    case ROLE_ADJ_TRIAL: {
                        float gg;
                        const float xo = xin[idx];
                        if (do_conv) {
                            gg = v;
                            if (VAR && want_sy) {             // before g and x_{k-1} are overwritten
                                const float s = xo - T.ctx.x[cur ^ 1][idx];
                                loc_sy = fmaf(s, fmaf(lamf, s, v - out[idx]), loc_sy);
                            }
                            out[idx] = gg;
                        } else {
                            gg = T.ctx.g[idx];
                        }
                        const float gt = VAR ? fmaf(lamf, xo, gg) : gg;   // grad f = A^T r + lambda x
                        const float xn = fmaxf(fmaf(-delta, gt, xo), 0.f);
                        T.ctx.x[cur ^ 1][idx] = xn;
                        store_shadow<KIND>(T.sh_out_hi[cur ^ 1], T.sh_out_lo[cur ^ 1], sidx, xn);
                        const float d = xn - xo;
                        loc = fmaf(d, d, loc);
                        if (VAR) {
                            loc_a = fmaf(gt, d, loc_a);
                            loc_x = fmaf(xn, xn, loc_x);
                        }
                        break;
                    }
                    default:
                        break;
                    }
                }
            }
        }
        if (!ok && lane == 0) fail();
    }

    // ---------------- block partial of the norm, teardown
    constexpr int NR = VAR ? 4 : 1;                // sums reduced per block
    __shared__ double s_red[NR][kThreads / 32];
    if (role == ROLE_FWD_INIT || role == ROLE_FWD_TRIAL || role == ROLE_ADJ_TRIAL) {
        double v[4] = {(double)loc, (double)loc_a, (double)loc_x, (double)loc_sy};
#pragma unroll
        for (int k = 0; k < NR; k++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
            if (lane == 0) s_red[k][warp] = v[k];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0 && (role == ROLE_FWD_INIT || role == ROLE_FWD_TRIAL || role == ROLE_ADJ_TRIAL)) {
        double t[NR];
        for (int k = 0; k < NR; k++) t[k] = 0.0;
        for (int i = 0; i < kThreads / 32; i++)
            for (int k = 0; k < NR; k++) t[k] += s_red[k][i];
        double* part = (role == ROLE_ADJ_TRIAL) ? T.ctx.part_m : T.ctx.part_f;
        part[blockIdx.x] = t[0];
        if (VAR) {
            if (want_a) T.ctx.part_a[blockIdx.x] = t[NR > 1 ? 1 : 0];
            if (want_x) T.ctx.part_x[blockIdx.x] = t[NR > 2 ? 2 : 0];
            if (want_sy) T.ctx.part_sy[blockIdx.x] = t[NR > 3 ? 3 : 0];
        }
    }
    if (run && warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tcols));
    }
}

// Launch helpers shared by the two translation units (VAR = false here in conv_tc.cu, VAR = true in
// conv_tc_var.cu).
template <bool VAR>
static cudaError_t tc_prepare_kinds(int kind)
{
    const int smax = 220 * 1024;
    auto set = [&](const void* f) { return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smax); };
    switch (kind) {
    case CDV_MODE_BF16: {
        cudaError_t e = set((const void*)conv_tc_kernel<CDV_MODE_BF16, 8, VAR>);
        return e == cudaSuccess ? set((const void*)conv_tc_kernel<CDV_MODE_BF16, 16, VAR>) : e;
    }
    case CDV_MODE_TF32: {
        cudaError_t e = set((const void*)conv_tc_kernel<CDV_MODE_TF32, 8, VAR>);
        return e == cudaSuccess ? set((const void*)conv_tc_kernel<CDV_MODE_TF32, 16, VAR>) : e;
    }
    case CDV_MODE_SPLIT_BF16X3: {
        cudaError_t e = set((const void*)conv_tc_kernel<CDV_MODE_SPLIT_BF16X3, 8, VAR>);
        return e == cudaSuccess ? set((const void*)conv_tc_kernel<CDV_MODE_SPLIT_BF16X3, 16, VAR>) : e;
    }
    default: return cudaErrorInvalidValue;
    }
}

template <int KIND, bool VAR>
static void tc_launch_kind(const TcArgs& t, const CUtensorMap* maps, size_t smem, cudaStream_t s)
{
    const dim3 grid((unsigned)t.grid);
    if (t.W == 8)
        conv_tc_kernel<KIND, 8, VAR><<<grid, kThreads, smem, s>>>(t, maps[0], maps[1], maps[2], maps[3]);
    else
        conv_tc_kernel<KIND, 16, VAR><<<grid, kThreads, smem, s>>>(t, maps[0], maps[1], maps[2], maps[3]);
}

template <bool VAR>
static cudaError_t tc_launch_kinds(const TcArgs& t, const CUtensorMap* maps, cudaStream_t s)
{
    const size_t smem = tc_smem_bytes(t);
    switch (t.kind) {
    case CDV_MODE_BF16: tc_launch_kind<CDV_MODE_BF16, VAR>(t, maps, smem, s); break;
    case CDV_MODE_TF32: tc_launch_kind<CDV_MODE_TF32, VAR>(t, maps, smem, s); break;
    case CDV_MODE_SPLIT_BF16X3: tc_launch_kind<CDV_MODE_SPLIT_BF16X3, VAR>(t, maps, smem, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace cdv

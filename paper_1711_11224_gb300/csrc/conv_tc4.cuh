// Tensor-core (tcgen05) direct convolution, narrow form: 4 output columns per tile and a sliding
// window of 32 output-plane slots.
//
// Same sums as conv_tc.cuh (out[s] = sum_j w[j] in[s + o - j], the forward of Property 1 with
// in = X, o = 0, w = H, the adjoint of Property 2 with in = R, o = 2p, w = H~), mapped so that the
// tensor pipe executes fewer zero products:
//  * Toeplitz operand along the contiguous axis with W = 4 output columns: the window of the 4
//    columns is 4 + q3 - 1 input columns, 24 (three 16-byte chunks) for q3 = 21, against 32 for 8
//    columns, so K / q3 falls from 32/21 to 24/21.  The window must start on a 16-byte chunk; every
//    second column group starts 4 columns off, so every input shadow exists twice, as stored (copy 0)
//    and shifted right by 4 columns (copy 1), and a tile reads the copy in which its window is aligned.
//  * An odd number of chunks per template row is paired across rows: one MMA K step of 16 takes two
//    chunks from anywhere in the staged input plane (the descriptor's leading-byte offset is the
//    distance between them), e.g. the last chunk of row j2 and the first of row j2 + 1.
//  * N = 4 columns x 32 slots = 128.  Output plane s lives in slot s mod 32 while it is open.  Input
//    plane u reaches planes u - o1 .. u - o1 + q1 - 1 (q1 <= 31 slots, one slot free); their Toeplitz
//    tiles are the template planes in rotated order, fetched as one contiguous run from a doubled copy
//    ([version][group of 2 slots]: version 0 pairs template planes (2e, 2e+1), version 1 (2e+1, 2e+2),
//    so any rotation is a run of whole 8-row groups).  A tile is a chunk of 32-aligned output planes;
//    only at its ends does an input plane reach fewer slots, and there the slots in range are
//    contiguous, so the MMA narrows to them.  After input plane u the plane in its j1 = 0 slot is
//    complete: the epilogue stores it and frees the slot.
//  * Two-level accumulation, warp roles, persistent CTAs, two 128-row M tiles per CTA, bounded waits
//    and split-BF16x3 with the A operand reused from the collector buffer: as in conv_tc.cuh.
#pragma once

#include "conv_tc.cuh"

namespace cdv {

namespace {

constexpr int kW4 = 4;           // output columns per tile
constexpr int kSlots = 32;       // plane slots (N = kW4 x kSlots = 128)
// Warps: 0 stages the input planes (TMA) and owns TMEM, 1 issues the MMAs, 2-9 run the epilogue, 10
// stages the template (bulk copies); one thread issues all copies of each producer warp.
constexpr int kThreads4 = 352;
constexpr int kBWarp = 10;

// K step i of an input plane: chunks (j2, c) of items 2i and 2i + 1 of the sequence over template
// rows and window chunks (row-major; an odd total ends with a pad item whose B chunk is zero).  The
// chunk of (j2, c) starts at a16(j2, c) = (q2 - 1 - j2) + c * rows in 16-byte units of the staged plane.
// Returns the descriptor start (16-byte units) and leading-byte offset (16-byte units) and which item
// comes first (the one at the lower address, so the offset is positive).
struct StepA {
    int start, lbo;
    int first, second;   // item indices (second may be the pad item q2 * kc)
};
__host__ __device__ inline StepA tc4_step(int i, int q2, int kc, int rows)
{
    const int a = 2 * i, b = 2 * i + 1, nitems = q2 * kc;
    const int aa = (q2 - 1 - a / kc) + (a % kc) * rows;
    const int ab = b < nitems ? (q2 - 1 - b / kc) + (b % kc) * rows : aa + 1;
    StepA s;
    if (ab >= aa) {
        s.start = aa;
        s.lbo = ab - aa;
        s.first = a;
        s.second = b;
    } else {
        s.start = ab;
        s.lbo = aa - ab;
        s.first = b;
        s.second = a;
    }
    return s;
}

}  // namespace

// Shared-memory layout of one CTA of the narrow kernel (bytes).
struct Tc4Smem {
    size_t a_bytes, b_bytes, off_b, off_bar, off_stage, off_tab, total;
    __host__ __device__ static Tc4Smem make(const TcArgs& t)
    {
        Tc4Smem s;
        s.a_bytes = (size_t)t.kc * (t.flat ? t.fboxes * 32 : t.rows) * 16;   // one part of one input plane
        s.b_bytes = (size_t)(kSlots / 2) * (2 * t.spst) * 128;           // one part of one stage
        s.off_b = (size_t)t.na * t.nprec * s.a_bytes;
        s.off_bar = s.off_b + (size_t)t.ns * t.nprec * s.b_bytes;
        s.off_stage = s.off_bar + 512;
        s.off_tab = s.off_stage + (size_t)8 * 32 * kW4 * 4;                    // 32 x 4 floats per epilogue warp
        s.total = s.off_tab + (size_t)t.steps * 8;                             // A descriptor offsets per K step
        return s;
    }
};

// One tile of the narrow kernel: output planes [S1, s1_end) (S1 a multiple of 32), rows
// [S2, S2 + 256), columns [S3, S3 + 4), input planes [ulo, uhi]; par = the shadow copy in which the
// window of the tile starts on a chunk.
// Flat tiles (forward): M row f (of block f0 .. f0 + 255) is row f mod lp of flat group G = f / lp;
// groups 0 .. ngrp0 - 1 are the column groups gfirst0 + 2i of copy 0, the next ngrp1 those of copy 1;
// rows f >= nf (or rows >= b2) hold no outputs.
struct Tc4Tile {
    int64_t S1, S2, S3, s1_end, ulo, uhi;
    int par;
    int64_t f0, nf;      // flat tiles: first M row, M rows holding groups
    int x0;              // TMA column of window chunk 0 (of the first group of the copy, for flat tiles)
    __host__ __device__ static Tc4Tile make(const TcArgs& T, int4 d)
    {
        Tc4Tile c;
        const int t3 = d.z % T.tiles3;
        const int t2 = d.z / T.tiles3;
        const ConvGeom& G = T.g;
        c.S1 = d.x;
        c.s1_end = d.y;
        const int64_t lo = c.S1 + G.o1 - G.q1 + 1;
        c.ulo = lo > 0 ? lo : 0;
        const int64_t hi = c.s1_end - 1 + G.o1;
        c.uhi = hi < G.a1 - 1 ? hi : G.a1 - 1;
        if (T.flat) {
            c.par = 0;
            c.f0 = (int64_t)t3 * kM * kMT;
            c.nf = (int64_t)(T.ngrp[0] + T.ngrp[1]) * T.lp;
            c.S2 = 0;
            c.S3 = 0;
        } else {
            c.S2 = (int64_t)t2 * kM * kMT;
            c.S3 = (int64_t)t3 * kW4;
            const int64_t x = c.S3 + G.o3 - (G.q3 - 1);
            c.par = (int)(((x % 8) + 8) % 8) == 0 ? 0 : 1;
            c.f0 = 0;
            c.nf = 0;
        }
        c.x0 = (int)(c.S3 + G.o3 - (G.q3 - 1)) + (c.par ? 4 : 0);
        return c;
    }
    // M tiles (of 128 rows) of the tile that hold outputs
    __host__ __device__ int mtiles(const TcArgs& T) const
    {
        const int64_t left = T.flat ? nf - f0 : T.g.b2 - S2;
        const int64_t n = (left + kM - 1) / kM;
        return (int)(n < kMT ? n : kMT);
    }
    // output planes that input plane u reaches inside the tile: [slo, shi] (empty if slo > shi)
    __host__ __device__ void planes(const ConvGeom& G, int64_t u, int64_t& slo, int64_t& shi) const
    {
        slo = u - G.o1 > S1 ? u - G.o1 : S1;
        const int64_t h = u - G.o1 + G.q1 - 1;
        shi = h < s1_end - 1 ? h : s1_end - 1;
    }
    // Slots the MMA of input plane u covers: [k0, k0 + ns), both multiples of 4 (N multiple of 16).
    // The slots in range are contiguous unless they wrap past slot 31; then all 32 are covered.
    __host__ __device__ void mma_slots(const ConvGeom& G, int64_t u, int& k0, int& ns) const
    {
        int64_t slo, shi;
        planes(G, u, slo, shi);
        const int a = (int)(slo % kSlots), b = (int)(shi % kSlots);
        if (a <= b && shi - slo < kSlots) {
            k0 = a & ~3;
            ns = ((b | 3) + 1) - k0;
        } else {
            k0 = 0;
            ns = kSlots;
        }
    }
};

template <int KIND, bool VAR>
__global__ void __launch_bounds__(kThreads4, 1)
conv_tc4_kernel(const __grid_constant__ TcArgs T, const __grid_constant__ CUtensorMap m00,
                const __grid_constant__ CUtensorMap m01, const __grid_constant__ CUtensorMap m10,
                const __grid_constant__ CUtensorMap m11, const __grid_constant__ CUtensorMap s00,
                const __grid_constant__ CUtensorMap s01, const __grid_constant__ CUtensorMap s10,
                const __grid_constant__ CUtensorMap s11)
{
    // maps: m<buffer><part> for shadow copy 0, s<buffer><part> for copy 1 (shifted by 4 columns)
    constexpr int NPREC = (KIND == CDV_MODE_SPLIT_BF16X3) ? 2 : 1;
    constexpr int EPT = (KIND == CDV_MODE_TF32) ? 4 : 8;       // elements per 16-byte K chunk
    static_assert(EPT == 8, "the narrow kernel pairs 8-element chunks (BF16 forms)");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const Tc4Smem lay = Tc4Smem::make(T);
    const ConvGeom& G = T.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int role = T.role;
    int sel = 0, cur = 0;
    bool do_conv = true;
    float delta = 0.f, lamf = 0.f;
    bool want_a = false, want_x = false, want_sy = false;
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

    unsigned char* sA = sm;
    unsigned char* sB = sm + lay.off_b;
    const unsigned bar0 = su32(sm + lay.off_bar);
    auto A_FULL = [&](int i) { return bar0 + 8u * i; };
    // input buffer i free again = the MMAs of the plane that used it (and of partial i) complete
    auto A_EMPTY = [&](int i) { return bar0 + 8u * (2 + i); };
    auto B_FULL = [&](int i) { return bar0 + 8u * (4 + i); };
    auto B_EMPTY = [&](int i) { return bar0 + 8u * (20 + i); };
    auto ACC_FREE = [&](int i) { return bar0 + 8u * (38 + i); };
    const unsigned DRAIN = bar0 + 8u * 40;
    unsigned* tslot = reinterpret_cast<unsigned*>(sm + lay.off_bar + 384);
    volatile int* sflag = reinterpret_cast<volatile int*>(sm + lay.off_bar + 392);

    const int kt0 = T.toff[blockIdx.x], kt1 = T.toff[blockIdx.x + 1];   // this CTA's tiles
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
    const int gbytes = 2 * T.spst * 128;                  // one 8-row group of one stage (one part)
    auto fail = [&]() {
        *sflag = 1;
        atomicExch(T.err, (int)CDV_ERR_TIMEOUT);
    };

    if (run && (warp == 0 || warp == kBWarp) && lane == 0) {
        // ---------------- producers: input planes (warp 0) and template stages (warp 10), each walking
        // the same tiles and input planes
        const bool doA = warp == 0, doB = warp == kBWarp;
        int bs = 0, it = 0, nb = 0;
        unsigned bph = 0;
        int a_uses[2] = {0, 0};
        for (int kt = kt0; kt < kt1 && !*sflag; ++kt) {
            const Tc4Tile C = Tc4Tile::make(T, T.tlist[kt]);
            const int x0 = C.x0;                                       // a multiple of 8
            const int fch0 = T.flat ? (int)(C.f0 / T.lp) : 0;          // flat: group and row of M row f0
            const int fr0 = T.flat ? (int)(C.f0 - (int64_t)fch0 * T.lp) : 0;
            const int64_t v0 = C.S2 + G.o2 - (G.q2 - 1);
            const CUtensorMap* mh = C.par ? (sel ? &s10 : &s00) : (sel ? &m10 : &m00);
            const CUtensorMap* ml = C.par ? (sel ? &s11 : &s01) : (sel ? &m11 : &m01);
            const CUtensorMap* sh = sel ? &s10 : &s00;               // flat tiles: copy 1 (copy 0 is mh, ml)
            const CUtensorMap* sl = sel ? &s11 : &s01;
            // flat tiles: TMA column of window chunk 0 of the first group of each copy (multiples of 8)
            const int xg[2] = {4 * T.gfirst[0] + (int)G.o3 - (G.q3 - 1), 4 * T.gfirst[1] + (int)G.o3 - (G.q3 - 1) + 4};
            for (int64_t u = C.ulo; u <= C.uhi && !*sflag; ++u, ++it) {
                if (doA) {
                const int ab = it % T.na;
                if (!mbar_wait(A_EMPTY(ab), (unsigned)(((it / T.na) & 1) ^ 1), T.wait_cycles)) { fail(); break; }
                mbar_expect_tx(A_FULL(ab), (unsigned)(NPREC * lay.a_bytes));
                a_uses[ab] = it / T.na + 1;
                for (int p = 0; p < NPREC; p++) {
                    const CUtensorMap* mp = p ? ml : mh;
                    const unsigned dst = su32(sA + ((size_t)ab * NPREC + p) * lay.a_bytes);
                    if (T.flat) {
                        // window chunk c: the 32 fboxes rows from M row f0, each 32-row box (boxes never
                        // cross a group, lp and f0 being multiples of 32) read from the copy of its flat
                        // group, 8c columns right of the start of that group's window
                        for (int c = 0; c < T.kc; c++) {
                            int gg = fch0, R = fr0;
                            for (int k = 0; k < T.fboxes; k++) {
                                const int cp = gg >= T.ngrp[0] ? 1 : 0;
                                const CUtensorMap* mb = cp ? (p ? sl : sh) : mp;
                                tma3(dst + (unsigned)((c * T.fboxes + k) * 32 * 16), mb,
                                     xg[cp] + (gg - (cp ? T.ngrp[0] : 0) + c) * EPT, R + G.o2 - (G.q2 - 1), (int)u,
                                     A_FULL(ab));
                                R += 32;
                                if (R == T.lp) {
                                    R = 0;
                                    ++gg;
                                }
                            }
                        }
                    } else {
                        for (int c = 0; c < T.kc; c++)
                            for (int h = 0; h < 2; h++)
                                tma3(dst + (unsigned)((c * T.rows + h * half) * 16), mp, x0 + c * EPT,
                                     (int)(v0 + h * half), (int)u, A_FULL(ab));
                    }
                }
                }
                if (doB) {
                    int k0, nsl;
                    C.mma_slots(G, u, k0, nsl);
                    // rotation: the j1 = 0 plane u - o1 sits in slot r; slot pair g holds doubled-sequence
                    // entries 2g + 32 - r and 2g + 33 - r, i.e. version (r & 1), group gs + g
                    const int r = (int)((((u - G.o1) % kSlots) + kSlots) % kSlots);
                    const int ver = r & 1;
                    const int gs = ver ? (31 - r) / 2 : 16 - r / 2;
                    const int g0 = k0 / 2, ng = nsl / 2;
                    for (int t = 0; t < T.nst; t++) {
                        if (!mbar_wait(B_EMPTY(bs), bph ^ 1, T.wait_cycles)) { fail(); break; }
                        mbar_expect_tx(B_FULL(bs), (unsigned)(NPREC * ng * gbytes));
                        for (int p = 0; p < NPREC; p++) {
                            const unsigned char* src = reinterpret_cast<const unsigned char*>(T.bt[p]) +
                                                       (((size_t)t * 2 + ver) * kSlots + (size_t)(gs + g0)) * gbytes;
                            const unsigned dst =
                                su32(sB + ((size_t)bs * NPREC + p) * lay.b_bytes) + (unsigned)(g0 * gbytes);
                            bulk_g2s(dst, src, (unsigned)(ng * gbytes), B_FULL(bs));
                        }
                        ++nb;
                        if (++bs == T.ns) { bs = 0; bph ^= 1; }
                    }
                }
            }
        }
        for (int ab = 0; ab < T.na; ab++)
            if (a_uses[ab] > 0) mbar_wait(A_FULL(ab), (unsigned)((a_uses[ab] - 1) & 1));
        for (int k = 0; k < T.ns && k < nb; k++) {
            const int idx = nb - 1 - k;
            mbar_wait(B_FULL(idx % T.ns), (unsigned)((idx / T.ns) & 1));
        }
    } else if (run && warp == 1) {
        // ---------------- MMA issuer (whole warp, one elected lane issues: the descriptors stay
        // warp-uniform; a loop on one lane ran 30% slower)
        const unsigned sA16 = (su32(sA) & 0x3FFFFu) >> 4, sB16 = (su32(sB) & 0x3FFFFu) >> 4;
        const unsigned a_part16 = (unsigned)(lay.a_bytes >> 4), b_part16 = (unsigned)(lay.b_bytes >> 4);
        const uint64_t db0 = sdesc(0, 128, (unsigned)gbytes);
        // per K step: the A descriptor's leading-byte offset field and start (16-byte units), the same
        // for every input plane and tile
        uint64_t* tab = reinterpret_cast<uint64_t*>(sm + lay.off_tab);
        for (int i = lane; i < T.steps; i += 32) {
            const StepA sa = tc4_step(i, G.q2, T.kc, T.flat ? T.fboxes * 32 : T.rows);
            tab[i] = ((uint64_t)sa.lbo << 16) + (uint64_t)sa.start;
        }
        __syncwarp();
        const uint64_t da0 = sdesc(0, 0, 128);
        int bs = 0, it = 0;
        unsigned bph = 0;
        bool ok = true;
        for (int kt = kt0; kt < kt1 && ok; ++kt) {
            const Tc4Tile C = Tc4Tile::make(T, T.tlist[kt]);
            const int nmt = C.mtiles(T);
            for (int64_t u = C.ulo; u <= C.uhi; ++u, ++it) {
                const int b = it & 1;                // accumulator buffer and input-plane buffer (na = 2)
                bool w = it < 2 || mbar_wait(ACC_FREE(b), (unsigned)(((it >> 1) - 1) & 1), T.wait_cycles);
                w = w && mbar_wait(A_FULL(b), (unsigned)((it >> 1) & 1), T.wait_cycles);
                if (!__all_sync(0xffffffffu, w && !*sflag)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                int k0, nsl;
                C.mma_slots(G, u, k0, nsl);
                const unsigned n = (unsigned)(kW4 * nsl);
                const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((unsigned)(kM >> 4) << 24);
                const unsigned d = tmem + (unsigned)(b * kNT + k0 * kW4);
                const unsigned a_hi = sA16 + (unsigned)(b * NPREC) * a_part16;
                const unsigned a_lo = a_hi + (unsigned)(NPREC - 1) * a_part16;
                unsigned acc = 0;
                for (int t = 0; t < T.nst; t++) {
                    if (!__all_sync(0xffffffffu, mbar_wait(B_FULL(bs), bph, T.wait_cycles))) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const unsigned b_hi = sB16 + (unsigned)(bs * NPREC) * b_part16 + (unsigned)((k0 / 2) * gbytes / 16);
                    const uint64_t bh = db0 + b_hi, bl = db0 + b_hi + (unsigned)(NPREC - 1) * b_part16;
                    const int nks = min(T.spst, T.steps - t * T.spst);
                    for (int sl = 0; sl < nks; sl++) {
                        const uint64_t off = tab[t * T.spst + sl];
                        const uint64_t ah = da0 + off + a_hi, al = da0 + off + a_lo;
                        const uint64_t kb = (uint64_t)sl * 16;          // two 128-byte chunks per K step
#pragma unroll
                        for (int mt = 0; mt < kMT; mt++) {
                            if (mt >= nmt) break;
                            const uint64_t am = (uint64_t)(mt * kM);
                            mma_step<KIND>(d + (unsigned)(mt * 2 * kNT), ah + am, al + am, bh + kb, bl + kb, idesc, acc);
                        }
                        acc = 1u;
                    }
                    mma_commit_elect(B_EMPTY(bs));
                    if (++bs == T.ns) { bs = 0; bph ^= 1; }
                }
                if (!ok) break;
                // one commit tells both the producer (input buffer b free) and the epilogue (partial b
                // complete)
                mma_commit_elect(A_EMPTY(b));
            }
        }
        if (!ok && lane == 0) fail();
        mma_commit_elect(DRAIN);
        if (!__all_sync(0xffffffffu, mbar_wait(DRAIN, 0)) && lane == 0) fail();
    }

    // ---------------- epilogue (warps 2..9): one output row per thread, warpgroup g owns M tile g
    float loc = 0.f, loc_a = 0.f, loc_x = 0.f, loc_sy = 0.f;
    if (warp >= 2 && warp < kBWarp) {
        const int mt = (warp - 2) >> 2;
        const int quarter = warp & 3;
        float* stg = reinterpret_cast<float*>(sm + lay.off_stage) + (warp - 2) * 32 * kW4;
        bool ok = true;
        int it = 0;
        // fused epilogue of one complete output plane s1 of the tile: this thread's 4 values of row
        // (its lane) go through the warp's staging tile, so that each store instruction covers 8 rows x
        // 4 consecutive columns
        // Element k (of 4) of this lane in a stored plane: row k * 8 + lane / 4 of the warp's 32, column
        // lane % 4 of the tile (the staging tile's transposed order); -1 if it holds no output.
        auto locate = [&](const Tc4Tile& C, int64_t s1, int k, int64_t& idx, int64_t& i0, int64_t& i1) -> bool {
            const int rr = k * 8 + (lane >> 2), c = lane & 3;
            int64_t s2 = C.S2 + mt * kM + quarter * 32 + rr;
            int64_t s3 = C.S3 + c;
            if (T.flat) {
                const int f = (int)C.f0 + mt * kM + quarter * 32 + rr;
                if (f >= (int)C.nf) return false;
                const int gg = f / T.lp;
                s2 = f - gg * T.lp;
                // flat group gg: copy 0's groups, then copy 1's; the groups of one copy are 8 columns apart
                const int cp = gg >= T.ngrp[0] ? 1 : 0;
                s3 = 4 * (int64_t)T.gfirst[cp] + 8 * (int64_t)(gg - (cp ? T.ngrp[0] : 0)) + c;
            }
            if (s2 >= G.b2 || s3 >= G.b3) return false;
            const int64_t row = s1 * G.b2 + s2;
            idx = row * G.b3 + s3;
            i0 = row * T.sh_pitch + s3;
            i1 = row * T.sh_pitch1 + s3 + 4;
            return true;
        };
        // the input the fused epilogue reads for an element (y for the residual, x_k for the update)
        auto operand = [&](int64_t idx) -> float {
            if (role == ROLE_FWD_INIT || role == ROLE_FWD_TRIAL) return T.ctx.y[idx];
            if (role == ROLE_ADJ_TRIAL) return xin[idx];
            return 0.f;
        };
        // fused epilogue of one complete output plane s1 of the tile: this thread's 4 values of row
        // (its lane) go through the warp's staging tile, so that each store instruction covers 8 rows x
        // 4 consecutive columns; pre[] holds the operands if they were loaded ahead
        auto finish = [&](const Tc4Tile& C, int64_t s1, const float* v, const float* pre) {
            __syncwarp();
            reinterpret_cast<float4*>(stg)[lane] = make_float4(v[0], v[1], v[2], v[3]);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float val = stg[(k * 8 + (lane >> 2)) * 4 + (lane & 3)];
                int64_t idx, i0, i1;
                if (!locate(C, s1, k, idx, i0, i1)) continue;
                const float opd = pre ? pre[k] : operand(idx);
                switch (role) {
                case ROLE_PLAIN:
                    out[idx] = val;
                    break;
                case ROLE_FWD_INIT:
                case ROLE_FWD_TRIAL: {
                    const float rr2 = val - opd;
                    out[idx] = rr2;
                    store_shadow<KIND>(T.sh_out_hi[sel], T.sh_out_lo[sel], i0, rr2);
                    store_shadow<KIND>(T.sh_out_hi1[sel], T.sh_out_lo1[sel], i1, rr2);
                    loc = fmaf(rr2, rr2, loc);
                    break;
                }
                case ROLE_ADJ_TRIAL: {
                    float gg;
                    const float xo = opd;
                    if (do_conv) {
                        gg = val;
                        if (VAR && want_sy) {
                            const float sd = xo - T.ctx.x[cur ^ 1][idx];
                            loc_sy = fmaf(sd, fmaf(lamf, sd, val - out[idx]), loc_sy);
                        }
                        out[idx] = gg;
                    } else {
                        gg = T.ctx.g[idx];
                    }
                    const float gt = VAR ? fmaf(lamf, xo, gg) : gg;
                    const float xn = fmaxf(fmaf(-delta, gt, xo), 0.f);
                    T.ctx.x[cur ^ 1][idx] = xn;
                    store_shadow<KIND>(T.sh_out_hi[cur ^ 1], T.sh_out_lo[cur ^ 1], i0, xn);
                    store_shadow<KIND>(T.sh_out_hi1[cur ^ 1], T.sh_out_lo1[cur ^ 1], i1, xn);
                    const float dd = xn - xo;
                    loc = fmaf(dd, dd, loc);
                    if (VAR) {
                        loc_a = fmaf(gt, dd, loc_a);
                        loc_x = fmaf(xn, xn, loc_x);
                    }
                    break;
                }
                default:
                    break;
                }
            }
        };
        for (int kt = kt0; kt < kt1 && ok; ++kt) {
            const Tc4Tile C = Tc4Tile::make(T, T.tlist[kt]);
            const bool rows_in = mt < C.mtiles(T);
            float tot[kSlots][kW4];
#pragma unroll
            for (int i = 0; i < kSlots; i++)
#pragma unroll
                for (int c = 0; c < kW4; c++) tot[i][c] = 0.f;
            if (!run) {
                // a retried trial reuses the stored gradient: only the update, for every plane of the tile
                if (!do_conv && rows_in && *(volatile int*)T.err == 0)
                    for (int64_t s1 = C.S1; s1 < C.s1_end; ++s1) finish(C, s1, &tot[0][0], nullptr);
                continue;
            }
            for (int64_t u = C.ulo; u <= C.uhi; ++u, ++it) {
                const int b = it & 1;
                // the plane completed by u (before the last input plane: only u - o1) and its operands,
                // loaded while the MMAs of u run
                const int64_t sdone = u - G.o1;
                const bool one = rows_in && u < G.a1 - 1 && sdone >= C.S1 && sdone < C.s1_end;
                float pre[4] = {0.f, 0.f, 0.f, 0.f};
                if (one) {
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        int64_t idx, i0, i1;
                        if (locate(C, sdone, k, idx, i0, i1)) pre[k] = operand(idx);
                    }
                }
                bool w = mbar_wait(A_EMPTY(b), (unsigned)((it >> 1) & 1), T.wait_cycles);   // plane it's MMAs done
                w = __all_sync(0xffffffffu, w && !*sflag);
                if (!w) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                int64_t slo, shi;
                C.planes(G, u, slo, shi);
                if (rows_in) {
                    // slot k holds plane slo + ((k - slo) mod 32) while it is open
                    const int klo = (int)(slo % kSlots);
                    const int span = (int)(shi - slo);
#pragma unroll
                    for (int qd = 0; qd < kSlots / 4; qd++) {             // 4 slots (16 columns) per load
                        bool vk[4];
#pragma unroll
                        for (int e = 0; e < 4; e++) vk[e] = ((4 * qd + e - klo + kSlots) % kSlots) <= span;
                        if (!vk[0] && !vk[1] && !vk[2] && !vk[3]) continue;    // warp-uniform
                        float v[16];
                        tmem_ld<16>(tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)((mt * 2 + b) * kNT + 4 * qd * kW4), v);
#pragma unroll
                        for (int e = 0; e < 4; e++)
#pragma unroll
                            for (int c = 0; c < kW4; c++)
                                if (vk[e]) tot[4 * qd + e][c] += v[kW4 * e + c];
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(ACC_FREE(b));
                if (!rows_in) continue;
                // planes complete after u: u - o1 (its last input plane), and at the volume's last input
                // plane every plane still open
                const int64_t first = u - G.o1 > C.S1 ? u - G.o1 : C.S1;
                const int64_t last = (u == G.a1 - 1) ? C.s1_end - 1 : (u - G.o1 < C.s1_end ? u - G.o1 : C.S1 - 1);
                for (int64_t s1 = first; s1 <= last; ++s1) {
                    if (s1 < u - G.o1) continue;
                    const int ks = (int)(s1 % kSlots);
                    float v[kW4];
#pragma unroll
                    for (int c = 0; c < kW4; c++) v[c] = 0.f;
#pragma unroll
                    for (int k = 0; k < kSlots; k++)
                        if (k == ks) {
#pragma unroll
                            for (int c = 0; c < kW4; c++) {
                                v[c] = tot[k][c];
                                tot[k][c] = 0.f;
                            }
                        }
                    finish(C, s1, v, one ? pre : nullptr);
                }
            }
        }
        if (!ok && lane == 0) fail();
    }

    // ---------------- block partials of the norms, teardown (as in conv_tc.cuh)
    constexpr int NR = VAR ? 4 : 1;
    __shared__ double s_red[NR][kThreads4 / 32];
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
        for (int i = 0; i < kThreads4 / 32; i++)
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

// Launch helpers shared by conv_tc4.cu (VAR = false) and conv_tc4_var.cu (VAR = true).
template <bool VAR>
static cudaError_t tc4_prepare_kinds(int kind)
{
    const int smax = 220 * 1024;
    auto set = [&](const void* f) { return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smax); };
    switch (kind) {
    case CDV_MODE_BF16: return set((const void*)conv_tc4_kernel<CDV_MODE_BF16, VAR>);
    case CDV_MODE_SPLIT_BF16X3: return set((const void*)conv_tc4_kernel<CDV_MODE_SPLIT_BF16X3, VAR>);
    default: return cudaSuccess;                 // TF32 runs the wide kernel only
    }
}

template <bool VAR>
static cudaError_t tc4_launch_kinds(const TcArgs& t, const CUtensorMap* m, cudaStream_t s)
{
    const size_t smem = Tc4Smem::make(t).total + 1024;
    const dim3 grid((unsigned)t.grid);
    switch (t.kind) {
    case CDV_MODE_BF16:
        conv_tc4_kernel<CDV_MODE_BF16, VAR><<<grid, kThreads4, smem, s>>>(t, m[0], m[1], m[2], m[3], m[4], m[5], m[6], m[7]);
        break;
    case CDV_MODE_SPLIT_BF16X3:
        conv_tc4_kernel<CDV_MODE_SPLIT_BF16X3, VAR><<<grid, kThreads4, smem, s>>>(t, m[0], m[1], m[2], m[3], m[4], m[5], m[6],
                                                                                 m[7]);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace cdv

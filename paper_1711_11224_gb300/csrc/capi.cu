// C ABI of libcdv: plans, the forward/adjoint operators, the template
// gradient, the projected-gradient iteration and Richardson-Lucy.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include <cuda.h>

#include "cdv_internal.h"

using namespace cdv;

namespace {

thread_local std::string g_err;

cdv_status fail(cdv_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

cdv_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(CDV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CDV_CUDA(call, what)                            \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr int kHistCap = 65536;

}  // namespace

void cdv::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

struct cdv_plan {
    int device = 0;
    int n = 0;
    int64_t m[3] = {1, 1, 1};
    int p[3] = {0, 0, 0};
    int q[3] = {1, 1, 1};
    cdv_mode mode = CDV_MODE_FP32;
    int64_t nx = 0, ny = 0, nh = 0;
    ConvGeom gf{}, ga{};
    ConvTile tf{}, ta{};
    float* H = nullptr;
    float* Ht = nullptr;
    double* absum = nullptr;
    bool has_psf = false;
    float* xw = nullptr;
    float* r0 = nullptr;
    float* r1 = nullptr;
    float* g = nullptr;
    float* ydev = nullptr;
    float* xdev = nullptr;
    float* aux = nullptr;
    double* part_f = nullptr;
    double* part_m = nullptr;
    double* part_a = nullptr;
    double* part_x = nullptr;
    double* part_sy = nullptr;
    int nparts = 0;
    IterState* st = nullptr;
    double* f_hist = nullptr;
    double* d_hist = nullptr;
    GradPsfPlan gp{};
    double* gp_part = nullptr;
    // tensor-core modes
    TcArgs tcf{}, tca{};            // forward / adjoint launch templates
    void* xsh[2][2] = {};           // BF16/TF32 shadows of the iterates [buffer][part]
    void* rsh[2][2] = {};           // shadows of the residuals
    void* xsh1[2][2] = {};          // narrow kernel: the same shifted right by 4 columns
    void* rsh1[2][2] = {};
    int64_t pitch_x = 0, pitch_r = 0, pitch_x1 = 0, pitch_r1 = 0;
    CUtensorMap map_x[8], map_r[8]; // hi0, lo0, hi1, lo1 of copy 0, then of copy 1 (narrow kernel)
    std::vector<int4> tc4_list[2];  // narrow kernel: host copy of the tile lists (forward, adjoint)
    int* dev_err = nullptr;
    bool tc() const { return mode == CDV_MODE_BF16 || mode == CDV_MODE_TF32 || mode == CDV_MODE_SPLIT_BF16X3; }
    bool fft() const { return mode == CDV_MODE_FFT; }
    FftPlan fftp{};
    bool sep() const { return mode == CDV_MODE_SEPARABLE; }
    SepPlan sepp{};
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    struct Key {
        const float* y;
        float* x;
        int K;
        int policy, max_halvings, max_rejects;
        double delta0, beta, tikhonov, armijo;
        int bb, pad_;
    } key{};
    bool key_valid = false;
    size_t bytes = 0;
    std::vector<void*> allocs;

    template <class T>
    cudaError_t alloc(T** ptr, size_t count)
    {
        void* v = nullptr;
        cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
        if (e != cudaSuccess) return e;
        allocs.push_back(v);
        bytes += count * sizeof(T);
        *ptr = static_cast<T*>(v);
        return cudaSuccess;
    }
    void release()
    {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
        fft_release(fftp);
        for (void* v : allocs) cudaFree(v);
        allocs.clear();
        if (cap) cudaStreamDestroy(cap);
        cap = nullptr;
    }
};

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

static int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Modelled tensor-pipe cycles of one direction for W output columns per plane (P = 128 / W planes
// per CTA): per tile and input plane, q2 x (K / 16) MMAs of N = W x (planes reached), each about
// max(46, N / 2) cycles; K = W + q3 - 1 + e rounded up to 16.
static double tc_model_cycles(const ConvGeom& g, int W, int e)
{
    const int P = 128 / W;
    const int K = (e + g.q3 + W - 1 + 15) / 16 * 16;
    double per_tile = 0.0;
    for (int v = -(g.q1 - 1); v < P; v++) {                       // input plane relative to the tile
        int nv = 0;
        for (int i = 0; i < P; i++) nv += (i - v >= 0 && i - v < g.q1) ? 1 : 0;
        if (nv == 0) continue;
        const int nn = W * (nv + ((W == 8 && (nv & 1)) ? 1 : 0));
        per_tile += std::max(46.0, nn / 2.0);
    }
    const double tiles = (double)ceil_div(g.b1, P) * ceil_div(g.b2, 256) * ceil_div(g.b3, W);
    return tiles * per_tile * g.q2 * (K / 16);
}

// Launch template of the tensor-core engine for one direction.
static bool tc_config(const cdv_plan* P, const ConvGeom& g, bool fwd, TcArgs& t)
{
    const int ept = (P->mode == CDV_MODE_TF32) ? 4 : 8;
    t = TcArgs{};
    t.g = g;
    t.kind = (int)P->mode;
    t.nprec = (P->mode == CDV_MODE_SPLIT_BF16X3) ? 2 : 1;
    const int off = g.o3 - (g.q3 - 1);
    t.e = ((off % ept) + ept) % ept;
    t.W = tc_model_cycles(g, 8, t.e) < tc_model_cycles(g, 16, t.e) ? 8 : 16;
    t.P = 128 / t.W;
    t.K = (t.e + g.q3 + t.W - 1 + 15) / 16 * 16;
    t.kchunks = t.K / ept;
    t.MT = 2;
    t.rows = (128 * t.MT + g.q2 - 1 + 15) / 16 * 16;
    t.tiles1 = ceil_div(g.b1, t.P);
    t.tiles2 = ceil_div(g.b2, 128 * t.MT);
    t.tiles3 = ceil_div(g.b3, t.W);
    const int64_t ntiles = (int64_t)t.tiles1 * t.tiles2 * t.tiles3;
    if (ntiles > (1LL << 31) - 1 || t.rows / 2 > 256 || t.K > 256) return false;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
        return false;
    t.ntiles = (int)ntiles;
    t.grid = (int)std::min<int64_t>(ntiles, nsm);     // one CTA per SM (about 220 KB of shared memory each)
    t.tmem_cols = 512;                      // 2 partial buffers x 2 M tiles x 128 columns
    t.sh_pitch = fwd ? P->pitch_r : P->pitch_x;
    t.err = P->dev_err;
    t.wait_cycles = kTcWaitCycles;
    // deepest template-tile ring that fits: each stage is one template row of one input plane
    t.na = 2;
    t.ns = 16;
    while (tc_smem_bytes(t) > 220 * 1024 && t.ns > 2) t.ns--;
    if (tc_smem_bytes(t) > 220 * 1024) t.na = 1;
    return tc_smem_bytes(t) <= 220 * 1024;
}

// Makespan of the wide kernel's persistent CTAs under the same MMA cost model, per 128-row M tile.
static double tc_wide_makespan(const TcArgs& t)
{
    const ConvGeom& g = t.g;
    std::vector<double> cta(std::max(1, t.grid), 0.0);
    std::vector<double> plane_cost(t.tiles1, 0.0);
    for (int t1 = 0; t1 < t.tiles1; t1++) {
        const int64_t S1 = (int64_t)t1 * t.P, s1_end = std::min<int64_t>(S1 + t.P, g.b1);
        const int64_t ulo = std::max<int64_t>(0, S1 + g.o1 - g.q1 + 1);
        const int64_t uhi = std::min<int64_t>(g.a1 - 1, s1_end - 1 + g.o1);
        for (int64_t u = ulo; u <= uhi; u++) {
            const int64_t ilo = std::max<int64_t>(0, u - g.o1 - S1);
            const int64_t ihi = std::min<int64_t>(s1_end - 1 - S1, u - g.o1 + g.q1 - 1 - S1);
            int64_t nv = ihi - ilo + 1;
            if (t.W == 8 && (nv & 1)) nv++;
            plane_cost[t1] += std::max(46.0, t.W * nv / 2.0);
        }
    }
    for (int tile = 0; tile < t.ntiles; tile++) {
        const int t2 = (tile / t.tiles3) % t.tiles2, t1 = tile / (t.tiles3 * t.tiles2);
        const int64_t nmt = std::min<int64_t>(t.MT, (g.b2 - (int64_t)t2 * 128 * t.MT + 127) / 128);
        cta[tile % cta.size()] += plane_cost[t1] * g.q2 * (t.K / 16) * (double)nmt;
    }
    return *std::max_element(cta.begin(), cta.end());
}

// Narrow-kernel template of one direction from the wide one (shared fields), with pc output planes
// per tile; false if the direction cannot run it (TF32, q1 > 31, windows not 4-column aligned, or
// too little shared memory).
static bool tc4_config(const cdv_plan* P, const TcArgs& wide, bool flat, TcArgs& t)
{
    const ConvGeom& g = wide.g;
    const int pc = 32;                       // tile lists cut the planes into 32-aligned ranges (tc4_partition)
    if (P->mode == CDV_MODE_TF32 || g.q1 > 31 || ((g.o3 - (g.q3 - 1)) % 4 + 4) % 4 != 0) return false;
    t = wide;
    t.w4 = 1;
    t.W = 4;
    t.P = 0;
    t.e = 0;
    t.pc = pc;
    t.kc = (g.q3 + 3 + 7) / 8;
    t.K = 8 * t.kc;
    t.kchunks = t.kc;
    t.steps = (g.q2 * t.kc + 1) / 2;
    if (2 * t.rows + 1 >= (1 << 14)) return false;                 // descriptor offsets (16-byte units)
    t.tiles1 = ceil_div(g.b1, pc);
    t.tiles2 = ceil_div(g.b2, 128 * t.MT);
    t.tiles3 = ceil_div(g.b3, 4);
    t.flat = 0;
    if (flat) {
        // the forward of a full convolution (o2 = 0, b2 = a2 + q2 - 1): rows that spill past a group's
        // lp rows read the next group's leading rows, which are zero, so M can run across groups
        if (g.o2 != 0 || g.b2 != g.a2 + g.q2 - 1) return false;
        t.flat = 1;
        t.lp = (int)((g.b2 + 31) / 32 * 32);
        for (int c = 0; c < 2; c++) {
            t.ngrp[c] = 0;
            t.gfirst[c] = -1;
        }
        for (int gi = 0; gi < t.tiles3; gi++) {
            const int64_t x = 4 * (int64_t)gi + g.o3 - (g.q3 - 1);
            const int c = (((x % 8) + 8) % 8) == 0 ? 0 : 1;
            if (t.gfirst[c] < 0) t.gfirst[c] = gi;
            t.ngrp[c]++;
        }
        for (int c = 0; c < 2; c++)
            if (t.gfirst[c] < 0) t.gfirst[c] = 0;
        t.nblk = (int)ceil_div((int64_t)(t.ngrp[0] + t.ngrp[1]) * t.lp, 128 * t.MT);
        // staged rows: per window chunk c, the 256 M rows shifted by c groups (c lp rows) plus q2 - 1
        // row shifts, in 32-row boxes; the rows between the chunks' windows are not loaded
        t.fboxes = ceil_div(128 * t.MT + g.q2 - 1, 32);
        if ((int64_t)t.kc * t.fboxes * 32 + g.q2 >= (1 << 14)) return false;     // descriptor offsets
        t.tiles2 = 1;
        t.tiles3 = t.nblk;
        if ((int64_t)(t.ngrp[0] + t.ngrp[1]) * t.lp >= (1LL << 30)) return false;
    }
    const int64_t ntiles = (int64_t)t.tiles1 * t.tiles2 * t.tiles3;
    if (ntiles > (1LL << 31) - 1) return false;
    t.ntiles = (int)ntiles;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
        return false;
    t.grid = (int)std::min<int64_t>(ntiles, nsm);
    t.na = 2;
    // template stages: as few per input plane as let two of them fit in shared memory (each stage
    // costs the MMA warp a wait and a commit and the producer its copies: on ring3d 8 K steps per stage
    // instead of 3 took split-BF16x3 from 7.56 to 6.61 ms per forward and adjoint, 16 instead of 3 BF16
    // from 5.44 to 3.82), the K steps spread evenly over them
    t.ns = 2;
    int most = 0;
    for (int sp = 1; sp <= t.steps; sp++) {
        t.spst = sp;
        if (tc4_smem_bytes(t) <= 220 * 1024) most = sp;
    }
    if (most == 0) return false;
    t.nst = (t.steps + most - 1) / most;
    t.spst = (t.steps + t.nst - 1) / t.nst;
    t.ns = 16;
    while (tc4_smem_bytes(t) > 220 * 1024 && t.ns > 2) t.ns--;
    return tc4_smem_bytes(t) <= 220 * 1024;
}

static cudaError_t make_map(CUtensorMap* m, const cdv_plan* P, void* base, int64_t d1, int64_t d2, int64_t d3,
                            int64_t pitch, int box_rows)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const bool tf = P->mode == CDV_MODE_TF32;
    const int es = tf ? 4 : 2, ept = tf ? 4 : 8;
    cuuint64_t dims[3] = {(cuuint64_t)d3, (cuuint64_t)d2, (cuuint64_t)d1};
    cuuint64_t strides[2] = {(cuuint64_t)(pitch * es), (cuuint64_t)(d2 * pitch * es)};
    cuuint32_t box[3] = {(cuuint32_t)ept, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor-core state of a plan: launch templates, shadows, tensor maps, tile storage.
static cudaError_t tc_setup(cdv_plan* P)
{
    cudaError_t e = tc_prepare((int)P->mode);
    if (e != cudaSuccess) return e;
    const int es = (P->mode == CDV_MODE_TF32) ? 4 : 2;
    const int nprec = (P->mode == CDV_MODE_SPLIT_BF16X3) ? 2 : 1;
    P->pitch_x = (P->m[2] + 7) / 8 * 8;
    P->pitch_r = (P->gf.b3 + 7) / 8 * 8;
    if (!tc_config(P, P->gf, true, P->tcf) || !tc_config(P, P->ga, false, P->tca)) return cudaErrorNotSupported;
    // The narrow kernel runs both directions or neither (each direction's epilogue writes the input
    // shadows of the other); CDV_TC_KERNEL=wide|narrow overrides the cycle model.
    {
        // narrow_rows / narrow_flat: the narrow kernel with the forward's M over rows only / over
        // (column group, row) whenever that is possible
        const char* env = getenv("CDV_TC_KERNEL");
        const bool force_wide = env && strcmp(env, "wide") == 0;
        const bool no_flat = env && strcmp(env, "narrow_rows") == 0, only_flat = env && strcmp(env, "narrow_flat") == 0;
        const bool force_narrow = env && (strcmp(env, "narrow") == 0 || no_flat || only_flat);
        TcArgs best[2];
        std::vector<int4> blist[2];
        std::vector<int> boff[2];
        double cost[2] = {-1.0, -1.0};
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
            nsm = 0;
        for (int d = 0; d < 2 && nsm > 0; d++) {
            const TcArgs& wide = d ? P->tca : P->tcf;
            for (int fl = 0; fl < (d == 0 ? 2 : 1); fl++) {
                TcArgs c;
                if ((fl && no_flat) || !tc4_config(P, wide, fl != 0, c)) continue;
                if (only_flat && d == 0 && !c.flat && tc4_config(P, wide, true, c)) continue;
                // the free cut (pc = 0) or chunk-major lists of pc planes (CDV_TC_DEAL=free|chunks
                // restricts the choice)
                const char* deal = getenv("CDV_TC_DEAL");
                for (int pc = 0; pc <= 512; pc += 32) {
                    if (deal && strcmp(deal, "free") == 0 && pc > 0) break;
                    if (deal && strcmp(deal, "chunks") == 0 && pc == 0) continue;
                    TcArgs cc = c;
                    std::vector<int4> L;
                    std::vector<int> O;
                    const double mk = tc4_partition(cc, nsm, pc, L, O);
                    if (cost[d] < 0.0 || mk < cost[d]) {
                        cost[d] = mk;
                        best[d] = cc;
                        blist[d] = L;
                        boff[d] = O;
                    }
                    if (pc >= wide.g.b1) break;
                }
            }
        }
        const bool legal = cost[0] >= 0.0 && cost[1] >= 0.0;
        const double wide_cost = tc_wide_makespan(P->tcf) + tc_wide_makespan(P->tca);
        if (legal && !force_wide && (force_narrow || cost[0] + cost[1] < wide_cost)) {
            P->tcf = best[0];
            P->tca = best[1];
            for (int d = 0; d < 2; d++) {
                TcArgs& t = d ? P->tca : P->tcf;
                int4* L = nullptr;
                int* O = nullptr;
                cudaError_t e2 = P->alloc(&L, blist[d].size());
                if (e2 == cudaSuccess) e2 = P->alloc(&O, boff[d].size());
                if (e2 == cudaSuccess)
                    e2 = cudaMemcpy(L, blist[d].data(), blist[d].size() * sizeof(int4), cudaMemcpyHostToDevice);
                if (e2 == cudaSuccess)
                    e2 = cudaMemcpy(O, boff[d].data(), boff[d].size() * sizeof(int), cudaMemcpyHostToDevice);
                if (e2 != cudaSuccess) return e2;
                t.tlist = L;
                t.toff = O;
                P->tc4_list[d] = blist[d];
            }
        }
    }
    const bool w4 = P->tcf.w4 != 0;
    P->pitch_x1 = (P->m[2] + 4 + 7) / 8 * 8;
    P->pitch_r1 = (P->gf.b3 + 4 + 7) / 8 * 8;
    if (w4) {
        // The narrow kernel's window chunks past an input's last column read zero columns stored in the
        // row pitch (its tensor maps span the whole pitch), not the TMA's out-of-bounds fill: loads
        // that ran past the right edge made the CTAs of the last column groups 20-30% slower.
        auto widen = [](int64_t& pitch, int64_t need) { pitch = std::max(pitch, (need + 7) / 8 * 8); };
        int64_t need[2][2];
        tc4_window_extent(P->tcf, need[0]);
        tc4_window_extent(P->tca, need[1]);
        widen(P->pitch_x, need[0][0]);
        widen(P->pitch_x1, need[0][1]);
        widen(P->pitch_r, need[1][0]);
        widen(P->pitch_r1, need[1][1]);
        P->tcf.sh_pitch = P->pitch_r;
        P->tca.sh_pitch = P->pitch_x;
    }
    const size_t xs = (size_t)P->m[0] * P->m[1] * P->pitch_x * es;
    const size_t rs = (size_t)P->gf.b1 * P->gf.b2 * P->pitch_r * es;
    for (int b = 0; b < 2; b++)
        for (int p = 0; p < 2; p++) {
            if (p < nprec) {
                if ((e = P->alloc((unsigned char**)&P->xsh[b][p], xs)) != cudaSuccess) return e;
                if ((e = P->alloc((unsigned char**)&P->rsh[b][p], rs)) != cudaSuccess) return e;
                // the columns past each row's data stay zero (nothing writes them)
                if (w4 && (e = cudaMemset(P->xsh[b][p], 0, xs)) != cudaSuccess) return e;
                if (w4 && (e = cudaMemset(P->rsh[b][p], 0, rs)) != cudaSuccess) return e;
            } else {
                P->xsh[b][p] = P->xsh[b][0];
                P->rsh[b][p] = P->rsh[b][0];
            }
        }
    if (w4) {
        // shifted copies: columns 0-3 of every row stay zero (the window left of column 0)
        const size_t xs1 = (size_t)P->m[0] * P->m[1] * P->pitch_x1 * es;
        const size_t rs1 = (size_t)P->gf.b1 * P->gf.b2 * P->pitch_r1 * es;
        for (int b = 0; b < 2; b++)
            for (int p = 0; p < 2; p++) {
                if (p < nprec) {
                    if ((e = P->alloc((unsigned char**)&P->xsh1[b][p], xs1)) != cudaSuccess) return e;
                    if ((e = P->alloc((unsigned char**)&P->rsh1[b][p], rs1)) != cudaSuccess) return e;
                    if ((e = cudaMemset(P->xsh1[b][p], 0, xs1)) != cudaSuccess) return e;
                    if ((e = cudaMemset(P->rsh1[b][p], 0, rs1)) != cudaSuccess) return e;
                } else {
                    P->xsh1[b][p] = P->xsh1[b][0];
                    P->rsh1[b][p] = P->rsh1[b][0];
                }
            }
    }
    // Toeplitz tiles: per part, q2 x kchunks x (q1*W rows) x 16 bytes (narrow kernel: its stages)
    for (int d = 0; d < 2; d++) {
        TcArgs& t = d ? P->tca : P->tcf;
        const size_t bytes = t.w4 ? tc4_btiles_bytes(t) : (size_t)P->q[1] * t.kchunks * P->q[0] * t.W * 16;
        for (int p = 0; p < 2; p++) {
            void* ptr = nullptr;
            if (p < nprec) {
                if ((e = P->alloc((unsigned char**)&ptr, bytes)) != cudaSuccess) return e;
            } else {
                ptr = const_cast<void*>(t.bt[0]);
            }
            t.bt[p] = ptr;
        }
    }
    for (int b = 0; b < 2; b++)
        for (int p = 0; p < 2; p++) {
            // the forward reads X through 32-row boxes in the flat layout, else through two boxes of half the
            // staged rows; the adjoint reads R through the latter
            const int bx = P->tcf.flat ? 32 : P->tcf.rows / 2, br = P->tca.rows / 2;
            // the narrow kernel's maps span the whole row pitch (zero columns past the data)
            const int64_t wx = w4 ? P->pitch_x : P->m[2], wr = w4 ? P->pitch_r : P->gf.b3;
            if ((e = make_map(&P->map_x[2 * b + p], P, P->xsh[b][p], P->m[0], P->m[1], wx, P->pitch_x, bx)) !=
                cudaSuccess)
                return e;
            if ((e = make_map(&P->map_r[2 * b + p], P, P->rsh[b][p], P->gf.b1, P->gf.b2, wr, P->pitch_r, br)) !=
                cudaSuccess)
                return e;
            if (!w4) continue;
            if ((e = make_map(&P->map_x[4 + 2 * b + p], P, P->xsh1[b][p], P->m[0], P->m[1], P->pitch_x1, P->pitch_x1,
                              bx)) != cudaSuccess)
                return e;
            if ((e = make_map(&P->map_r[4 + 2 * b + p], P, P->rsh1[b][p], P->gf.b1, P->gf.b2, P->pitch_r1, P->pitch_r1,
                              br)) != cudaSuccess)
                return e;
        }
    for (int b = 0; b < 2; b++) {
        P->tcf.sh_out_hi[b] = P->rsh[b][0];
        P->tcf.sh_out_lo[b] = P->rsh[b][1];
        P->tca.sh_out_hi[b] = P->xsh[b][0];
        P->tca.sh_out_lo[b] = P->xsh[b][1];
        P->tcf.sh_out_hi1[b] = P->rsh1[b][0];
        P->tcf.sh_out_lo1[b] = P->rsh1[b][1];
        P->tca.sh_out_hi1[b] = P->xsh1[b][0];
        P->tca.sh_out_lo1[b] = P->xsh1[b][1];
    }
    P->tcf.sh_pitch1 = P->pitch_r1;
    P->tca.sh_pitch1 = P->pitch_x1;
    P->nparts = std::max(P->nparts, std::max(P->tcf.grid, P->tca.grid));
    return cudaSuccess;
}

extern "C" {

const char* cdv_status_string(cdv_status s)
{
    switch (s) {
    case CDV_OK: return "CDV_OK";
    case CDV_ERR_INVALID_ARG: return "CDV_ERR_INVALID_ARG";
    case CDV_ERR_SHAPE: return "CDV_ERR_SHAPE";
    case CDV_ERR_UNSUPPORTED: return "CDV_ERR_UNSUPPORTED";
    case CDV_ERR_OOM: return "CDV_ERR_OOM";
    case CDV_ERR_CUDA: return "CDV_ERR_CUDA";
    case CDV_ERR_TIMEOUT: return "CDV_ERR_TIMEOUT";
    case CDV_ERR_NOT_DESCENDING: return "CDV_ERR_NOT_DESCENDING";
    case CDV_ERR_NONFINITE: return "CDV_ERR_NONFINITE";
    case CDV_ERR_NO_PSF: return "CDV_ERR_NO_PSF";
    }
    return "CDV_ERR_UNKNOWN";
}

const char* cdv_last_error(void) { return g_err.c_str(); }

int cdv_version(void) { return 100; }

void cdv_iter_opts_default(cdv_iter_opts* o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->x0_policy = CDV_X0_GIVEN;
    o->delta0 = 0.0;
    o->beta = 0.5;
    o->max_halvings = 20;
    o->max_rejects = 16;
    o->use_graph = 1;
}

static void* plan_alloc(void* owner, size_t bytes)
{
    unsigned char* v = nullptr;
    return static_cast<cdv_plan*>(owner)->alloc(&v, bytes) == cudaSuccess ? v : nullptr;
}

cdv_status cdv_plan_create(cdv_plan** out, int n, const int64_t* m, const int32_t* p, cdv_mode mode, void* stream)
{
    (void)stream;
    if (!out) return fail(CDV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!m || !p) return fail(CDV_ERR_INVALID_ARG, "m or p is NULL");
    if (n < 1 || n > 3) return fail(CDV_ERR_SHAPE, "n = %d, must be 1, 2 or 3", n);
    if (mode != CDV_MODE_FP32 && mode != CDV_MODE_BF16 && mode != CDV_MODE_TF32 && mode != CDV_MODE_SPLIT_BF16X3 &&
        mode != CDV_MODE_FFT && mode != CDV_MODE_SEPARABLE)
        return fail(CDV_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
    for (int i = 0; i < n; i++) {
        if (m[i] < 1) return fail(CDV_ERR_SHAPE, "m[%d] = %lld < 1", i, (long long)m[i]);
        if (p[i] < 0) return fail(CDV_ERR_SHAPE, "p[%d] = %d < 0", i, (int)p[i]);
        if (m[i] > (1LL << 31) || p[i] > (1 << 20)) return fail(CDV_ERR_SHAPE, "axis %d too large", i);
    }
    cdv_plan* P = new cdv_plan();
    P->n = n;
    P->mode = mode;
    for (int i = 0; i < n; i++) {
        P->m[3 - n + i] = m[i];
        P->p[3 - n + i] = p[i];
    }
    for (int i = 0; i < 3; i++) P->q[i] = 2 * P->p[i] + 1;
    double nxd = 1, nyd = 1;
    for (int i = 0; i < 3; i++) {
        nxd *= (double)P->m[i];
        nyd *= (double)(P->m[i] + 2 * P->p[i]);
    }
    if (nyd > 4.0e10) {
        delete P;
        return fail(CDV_ERR_SHAPE, "problem too large (%.3g samples)", nyd);
    }
    P->nx = P->m[0] * P->m[1] * P->m[2];
    P->ny = (P->m[0] + 2 * P->p[0]) * (P->m[1] + 2 * P->p[1]) * (P->m[2] + 2 * P->p[2]);
    P->nh = (int64_t)P->q[0] * P->q[1] * P->q[2];
    if (mode == CDV_MODE_FP32 && !conv_fp32_supported(P->q[2])) {     // the FFT comparator takes any width
        delete P;
        return fail(CDV_ERR_UNSUPPORTED, "template width %d along the contiguous axis: this build supports odd 1..31",
                    P->q[2]);
    }
    if (mode == CDV_MODE_SEPARABLE && !sep_supported(P->q)) {
        delete P;
        return fail(CDV_ERR_UNSUPPORTED, "separable template: this build supports odd 1..31 samples per axis");
    }
    P->gf = ConvGeom{P->m[0], P->m[1], P->m[2],
                     P->m[0] + 2 * P->p[0], P->m[1] + 2 * P->p[1], P->m[2] + 2 * P->p[2],
                     0, 0, 0, P->q[0], P->q[1], P->q[2]};
    P->ga = ConvGeom{P->gf.b1, P->gf.b2, P->gf.b3, P->m[0], P->m[1], P->m[2],
                     2 * P->p[0], 2 * P->p[1], 2 * P->p[2], P->q[0], P->q[1], P->q[2]};
    P->tf = conv_fp32_tile(P->gf);
    P->ta = conv_fp32_tile(P->ga);
    P->nparts = std::max(std::max(P->tf.grid, P->ta.grid), std::max(fft_epilogue_blocks(), sep_blocks()));
    P->gp = GradPsfPlan{P->m[0], P->m[1], P->m[2], P->q[0], P->q[1], P->q[2], 1, 1};

    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess && conv_fp32_supported(P->q[2])) e = conv_fp32_prepare(P->q[2]);
    if (e == cudaSuccess) e = grad_psf_prepare();
    if (e == cudaSuccess) P->gp.chunks = grad_psf_chunks(P->gp);
    if (e == cudaSuccess && small_supported(P->m, P->p)) {
        SmallRun r{};
        for (int i = 0; i < 3; i++) {
            r.m[i] = P->m[i];
            r.p[i] = P->p[i];
        }
        e = small_iterate(r, nullptr, true);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = P->alloc(&P->dev_err, 1);
    if (e == cudaSuccess) e = cudaMemset(P->dev_err, 0, sizeof(int));
    if (e == cudaSuccess && P->tc()) {
        e = tc_setup(P);
        if (e == cudaErrorNotSupported) {
            cudaGetLastError();
            P->release();
            delete P;
            return fail(CDV_ERR_UNSUPPORTED, "no tensor-core kernel for this size (template rows > 129 or too wide)");
        }
    }
    if (e == cudaSuccess && P->fft()) e = fft_setup(P->fftp, P->gf, plan_alloc, P);
    if (e == cudaSuccess && P->sep()) e = sep_setup(P->sepp, P->m, P->p, plan_alloc, P);
    if (e == cudaSuccess) e = P->alloc(&P->H, P->nh);
    if (e == cudaSuccess) e = P->alloc(&P->Ht, P->nh);
    if (e == cudaSuccess) e = P->alloc(&P->absum, 1);
    if (e == cudaSuccess) e = P->alloc(&P->xw, P->nx);
    if (e == cudaSuccess) e = P->alloc(&P->g, P->nx);
    if (e == cudaSuccess) e = P->alloc(&P->xdev, P->nx);
    if (e == cudaSuccess) e = P->alloc(&P->aux, P->nx);
    if (e == cudaSuccess) e = P->alloc(&P->r0, P->ny);
    if (e == cudaSuccess) e = P->alloc(&P->r1, P->ny);
    if (e == cudaSuccess) e = P->alloc(&P->ydev, P->ny);
    if (e == cudaSuccess) e = P->alloc(&P->part_f, P->nparts);
    if (e == cudaSuccess) e = P->alloc(&P->part_m, P->nparts);
    if (e == cudaSuccess) e = P->alloc(&P->part_a, P->nparts);
    if (e == cudaSuccess) e = P->alloc(&P->part_x, P->nparts);
    if (e == cudaSuccess) e = P->alloc(&P->part_sy, P->nparts);
    if (e == cudaSuccess) e = P->alloc(&P->st, 1);
    if (e == cudaSuccess) e = P->alloc(&P->f_hist, kHistCap + 1);
    if (e == cudaSuccess) e = P->alloc(&P->d_hist, kHistCap);
    if (e == cudaSuccess) e = P->alloc(&P->gp_part, grad_psf_partials(P->gp));
    if (e != cudaSuccess) {
        const bool oom = (e == cudaErrorMemoryAllocation);
        cudaGetLastError();
        P->release();
        delete P;
        return oom ? fail(CDV_ERR_OOM, "workspace allocation failed") : cuda_fail(e, "plan create");
    }
    *out = P;
    return CDV_OK;
}

cdv_status cdv_plan_workspace_size(const cdv_plan* plan, size_t* bytes)
{
    if (!plan || !bytes) return fail(CDV_ERR_INVALID_ARG, "NULL argument");
    *bytes = plan->bytes;
    return CDV_OK;
}

cdv_status cdv_plan_set_psf(cdv_plan* plan, const float* H, void* stream)
{
    if (!plan || !H) return fail(CDV_ERR_INVALID_ARG, "NULL argument");
    if (plan->sep())
        return fail(CDV_ERR_UNSUPPORTED, "a separable plan takes its template as per-axis factors "
                                         "(cdv_plan_set_psf_factors)");
    cudaStream_t s = (cudaStream_t)stream;
    CDV_CUDA(cudaMemcpyAsync(plan->H, H, plan->nh * sizeof(float), cudaMemcpyDeviceToDevice, s), "copy H");
    CDV_CUDA(launch_flip(plan->H, plan->Ht, plan->q[0], plan->q[1], plan->q[2], s), "flip H");
    CDV_CUDA(launch_abs_sum(plan->H, plan->nh, plan->absum, s), "sum |H|");
    if (plan->tc() && plan->tcf.w4) {
        CDV_CUDA(tc4_build_btiles(plan->tcf, plan->H, const_cast<void*>(plan->tcf.bt[0]),
                                  const_cast<void*>(plan->tcf.bt[1]), s), "Toeplitz stages (forward)");
        CDV_CUDA(tc4_build_btiles(plan->tca, plan->Ht, const_cast<void*>(plan->tca.bt[0]),
                                  const_cast<void*>(plan->tca.bt[1]), s), "Toeplitz stages (adjoint)");
    } else if (plan->tc()) {
        const int q3 = plan->q[2];
        CDV_CUDA(tc_build_btiles(plan->H, plan->q[0], plan->q[1], q3, q3 - 1 + plan->tcf.e, plan->tcf.K, plan->tcf.W,
                                 (int)plan->mode, const_cast<void*>(plan->tcf.bt[0]),
                                 const_cast<void*>(plan->tcf.bt[1]), s), "Toeplitz tiles (forward)");
        CDV_CUDA(tc_build_btiles(plan->Ht, plan->q[0], plan->q[1], q3, q3 - 1 + plan->tca.e, plan->tca.K, plan->tca.W,
                                 (int)plan->mode, const_cast<void*>(plan->tca.bt[0]),
                                 const_cast<void*>(plan->tca.bt[1]), s), "Toeplitz tiles (adjoint)");
    }
    if (plan->fft())
        CDV_CUDA(fft_set_psf(plan->fftp, plan->H, plan->q[0], plan->q[1], plan->q[2], s), "template spectrum");
    plan->has_psf = true;
    return CDV_OK;
}

cdv_status cdv_plan_set_psf_factors(cdv_plan* plan, const float* const* h, void* stream)
{
    if (!plan || !h) return fail(CDV_ERR_INVALID_ARG, "NULL argument");
    if (!plan->sep()) return fail(CDV_ERR_UNSUPPORTED, "per-axis factors need a CDV_MODE_SEPARABLE plan");
    const float* hp[3] = {nullptr, nullptr, nullptr};
    for (int i = 0; i < plan->n; i++) {
        if (!h[i]) return fail(CDV_ERR_INVALID_ARG, "factor %d is NULL", i);
        hp[3 - plan->n + i] = h[i];
    }
    cudaStream_t s = (cudaStream_t)stream;
    CDV_CUDA(sep_set_factors(plan->sepp, hp, plan->q, plan->H, s), "separable factors");
    CDV_CUDA(launch_flip(plan->H, plan->Ht, plan->q[0], plan->q[1], plan->q[2], s), "flip H");
    CDV_CUDA(launch_abs_sum(plan->H, plan->nh, plan->absum, s), "sum |H|");
    plan->has_psf = true;
    return CDV_OK;
}

cdv_status cdv_plan_lipschitz(const cdv_plan* plan, double* L)
{
    if (!plan || !L) return fail(CDV_ERR_INVALID_ARG, "NULL argument");
    if (!plan->has_psf) return fail(CDV_ERR_NO_PSF, "no template set");
    double a = 0.0;
    CDV_CUDA(cudaDeviceSynchronize(), "sync");
    CDV_CUDA(cudaMemcpy(&a, plan->absum, sizeof(double), cudaMemcpyDeviceToHost), "read sum |H|");
    *L = a * a;
    return CDV_OK;
}

// Tensor-pipe multiply-adds of one launch of the tensor-core engine: per plane tile, input plane,
// template row, K step and M tile one MMA of 128 x N x 16 per product, N = W x (planes covered,
// odd counts padded for W = 8) -- the loops of the kernel, counted on the host.
static double tc_executed_macs(const TcArgs& t)
{
    const ConvGeom& g = t.g;
    double n_sum = 0.0;
    for (int t1 = 0; t1 < t.tiles1; t1++) {
        const int64_t S1 = (int64_t)t1 * t.P, s1_end = std::min<int64_t>(S1 + t.P, g.b1);
        const int64_t ulo = std::max<int64_t>(0, S1 + g.o1 - g.q1 + 1);
        const int64_t uhi = std::min<int64_t>(g.a1 - 1, s1_end - 1 + g.o1);
        for (int64_t u = ulo; u <= uhi; u++) {
            const int64_t ilo = std::max<int64_t>(0, u - g.o1 - S1);
            const int64_t ihi = std::min<int64_t>(s1_end - 1 - S1, u - g.o1 + g.q1 - 1 - S1);
            int64_t nv = ihi - ilo + 1;
            if (t.W == 8 && (nv & 1)) nv++;
            n_sum += (double)(t.W * nv);
        }
    }
    double mtiles = 0.0;
    for (int t2 = 0; t2 < t.tiles2; t2++)
        mtiles += (double)std::min<int64_t>(t.MT, (g.b2 - (int64_t)t2 * 128 * t.MT + 127) / 128);
    const double products = (t.nprec == 2) ? 3.0 : 1.0;
    return n_sum * mtiles * 128.0 * t.K * g.q2 * t.tiles3 * products;
}

cdv_status cdv_plan_describe(const cdv_plan* plan, cdv_plan_info* out)
{
    if (!plan || !out) return fail(CDV_ERR_INVALID_ARG, "NULL argument");
    *out = cdv_plan_info{};
    out->mode = (int32_t)plan->mode;
    out->algorithmic_macs = (double)plan->nx * (double)plan->nh;
    for (int d = 0; d < 2; d++) {
        if (plan->fft()) {
            continue;
        } else if (plan->sep()) {
            out->grid[d] = sep_blocks();
            out->executed_macs[d] = sep_pass_macs(plan->sepp, d == 0);
        } else if (plan->mode == CDV_MODE_FP32) {
            const ConvTile& c = d ? plan->ta : plan->tf;
            out->grid[d] = c.grid;
            out->tiles[d] = c.grid;
            out->executed_macs[d] = out->algorithmic_macs;
        } else {
            const TcArgs& t = d ? plan->tca : plan->tcf;
            out->cols[d] = t.W;
            out->K[d] = t.K;
            out->grid[d] = t.grid;
            out->tiles[d] = t.ntiles;
            out->executed_macs[d] = t.w4 ? tc4_executed_macs(t, plan->tc4_list[d]) : tc_executed_macs(t);
        }
    }
    return CDV_OK;
}

cdv_status cdv_plan_destroy(cdv_plan* plan)
{
    if (!plan) return CDV_OK;
    plan->release();
    delete plan;
    return CDV_OK;
}

static cdv_status run_conv(cdv_plan* P, bool fwd, int batch, const float* in, float* out, cudaStream_t s)
{
    if (!in || !out) return fail(CDV_ERR_INVALID_ARG, "NULL array");
    if (batch < 1 || batch > 65535) return fail(CDV_ERR_INVALID_ARG, "batch = %d", batch);
    if (!P->has_psf) return fail(CDV_ERR_NO_PSF, "no template set");
    if (P->sep()) {
        for (int b = 0; b < batch; b++)
            CDV_CUDA(sep_conv(P->sepp, fwd, in + (int64_t)b * (fwd ? P->nx : P->ny),
                              out + (int64_t)b * (fwd ? P->ny : P->nx), s),
                     fwd ? "forward (separable)" : "adjoint (separable)");
        return CDV_OK;
    }
    if (P->fft()) {
        const ConvGeom& g = fwd ? P->gf : P->ga;
        for (int b = 0; b < batch; b++)
            CDV_CUDA(fft_conv(P->fftp, g, fwd, in + (int64_t)b * (fwd ? P->nx : P->ny),
                              out + (int64_t)b * (fwd ? P->ny : P->nx), s),
                     fwd ? "forward (FFT)" : "adjoint (FFT)");
        return CDV_OK;
    }
    if (P->tc()) {
        const ConvGeom& g = fwd ? P->gf : P->ga;
        for (int b = 0; b < batch; b++) {
            const float* src = in + (int64_t)b * (fwd ? P->nx : P->ny);
            if (fwd)
                CDV_CUDA(tc_shadow(src, g.a1 * g.a2, g.a3, P->pitch_x, (int)P->mode, P->xsh[0][0], P->xsh[0][1], s),
                         "input shadow");
            else
                CDV_CUDA(tc_shadow(src, g.a1 * g.a2, g.a3, P->pitch_r, (int)P->mode, P->rsh[0][0], P->rsh[0][1], s),
                         "input shadow");
            if (P->tcf.w4) {
                if (fwd)
                    CDV_CUDA(tc4_shadow1(src, g.a1 * g.a2, g.a3, P->pitch_x1, (int)P->mode, P->xsh1[0][0],
                                         P->xsh1[0][1], s), "input shadow (shifted)");
                else
                    CDV_CUDA(tc4_shadow1(src, g.a1 * g.a2, g.a3, P->pitch_r1, (int)P->mode, P->rsh1[0][0],
                                         P->rsh1[0][1], s), "input shadow (shifted)");
            }
            TcArgs t = fwd ? P->tcf : P->tca;
            t.role = ROLE_PLAIN;
            t.out = out + (int64_t)b * (fwd ? P->ny : P->nx);
            CDV_CUDA(tc_launch(t, fwd ? P->map_x : P->map_r, s), fwd ? "forward (tensor cores)" : "adjoint (tensor cores)");
        }
        return CDV_OK;
    }
    ConvLaunch L{};
    L.g = fwd ? P->gf : P->ga;
    L.in = in;
    L.out = out;
    L.w = fwd ? P->H : P->Ht;
    L.role = ROLE_PLAIN;
    L.batch = batch;
    L.in_bstride = fwd ? P->nx : P->ny;
    L.out_bstride = fwd ? P->ny : P->nx;
    CDV_CUDA(conv_fp32_launch(L, fwd ? P->tf : P->ta, s), fwd ? "forward" : "adjoint");
    return CDV_OK;
}

cdv_status cdv_forward(cdv_plan* plan, int batch, const float* X, float* Y, void* stream)
{
    if (!plan) return fail(CDV_ERR_INVALID_ARG, "plan is NULL");
    return run_conv(plan, true, batch, X, Y, (cudaStream_t)stream);
}

cdv_status cdv_adjoint(cdv_plan* plan, int batch, const float* R, float* G, void* stream)
{
    if (!plan) return fail(CDV_ERR_INVALID_ARG, "plan is NULL");
    return run_conv(plan, false, batch, R, G, (cudaStream_t)stream);
}

cdv_status cdv_grad_psf(cdv_plan* plan, int batch, const float* X, const float* dY, float* dH, void* stream)
{
    if (!plan || !X || !dY || !dH) return fail(CDV_ERR_INVALID_ARG, "NULL argument");
    if (batch < 1) return fail(CDV_ERR_INVALID_ARG, "batch = %d", batch);
    GradPsfPlan g = plan->gp;
    g.batch = batch;
    CDV_CUDA(launch_grad_psf(g, X, dY, plan->gp_part, dH, (cudaStream_t)stream), "grad_psf");
    return CDV_OK;
}

static IterCtx make_ctx(cdv_plan* P, const float* Y, float* X)
{
    IterCtx c{};
    c.x[0] = X;
    c.x[1] = P->xw;
    c.r[0] = P->r0;
    c.r[1] = P->r1;
    c.g = P->g;
    c.y = Y;
    c.aux = P->aux;
    c.part_f = P->part_f;
    c.part_m = P->part_m;
    c.part_a = P->part_a;
    c.part_x = P->part_x;
    c.part_sy = P->part_sy;
    c.st = P->st;
    c.f_hist = P->f_hist;
    c.d_hist = P->d_hist;
    return c;
}

// One projected-gradient run as three phases: 0 = prologue (x_0, state, initial forward and decision),
// 1 = one trial slot (adjoint + update, forward + residual, decision), 2 = epilogue (x_K into X).
struct RunCtx {
    cdv_plan* P;
    const float* Y;
    float* X;
    int K;
    cdv_iter_opts o;
};

static cdv_status run_phase(void* vctx, int phase, bool loop, unsigned long long h, cudaStream_t s)
{
    RunCtx& R = *static_cast<RunCtx*>(vctx);
    cdv_plan* P = R.P;
    const IterCtx c = make_ctx(P, R.Y, R.X);
    const int max_trials = R.K + R.o.max_rejects + 1;
    int nf, nm;
    if (P->fft()) {
        nf = nm = fft_epilogue_blocks();
    } else if (P->sep()) {
        nf = nm = sep_blocks();
    } else if (P->tc()) {
        nf = P->tcf.grid;
        nm = P->tca.grid;
    } else {
        nf = P->tf.grid;
        nm = P->ta.grid;
    }
    auto decide = [&](int init) -> cudaError_t {
        return loop ? launch_decide_loop(c, nf, init ? 0 : nm, init, h, max_trials, s)
                    : launch_decide(c, nf, init ? 0 : nm, init, s);
    };
    if (phase == 0) {
        CDV_CUDA(launch_x0(R.o.x0_policy, R.X, R.Y, P->m[0], P->m[1], P->m[2], P->p[0], P->p[1], P->p[2], s), "x0");
        if (P->tc())
            CDV_CUDA(tc_shadow(R.X, P->m[0] * P->m[1], P->m[2], P->pitch_x, (int)P->mode, P->xsh[0][0], P->xsh[0][1], s),
                     "x0 shadow");
        if (P->tc() && P->tcf.w4)
            CDV_CUDA(tc4_shadow1(R.X, P->m[0] * P->m[1], P->m[2], P->pitch_x1, (int)P->mode, P->xsh1[0][0],
                                 P->xsh1[0][1], s), "x0 shadow (shifted)");
        CDV_CUDA(launch_state_init(P->st, R.o.delta0, P->absum, R.o.beta, R.o.max_halvings, R.o.max_rejects, R.K,
                                   kHistCap, R.o.tikhonov, R.o.armijo, R.o.bb, s), "state");
        if (R.o.tikhonov != 0.0) CDV_CUDA(launch_sumsq(R.X, P->nx, P->part_x, s), "||x_0||^2");
        if (P->fft()) {
            CDV_CUDA(fft_role(P->fftp, P->gf, ROLE_FWD_INIT, c, s), "forward (initial, FFT)");
        } else if (P->sep()) {
            CDV_CUDA(sep_role(P->sepp, true, ROLE_FWD_INIT, c, s), "forward (initial, separable)");
        } else if (P->tc()) {
            TcArgs F = P->tcf;
            F.ctx = c;
            F.role = ROLE_FWD_INIT;
            CDV_CUDA(tc_launch(F, P->map_x, s), "forward (initial, tensor cores)");
        } else {
            ConvLaunch F{};
            F.g = P->gf;
            F.w = P->H;
            F.batch = 1;
            F.ctx = c;
            F.role = ROLE_FWD_INIT;
            CDV_CUDA(conv_fp32_launch(F, P->tf, s), "forward (initial)");
        }
        CDV_CUDA(decide(1), "decide (initial)");
    } else if (phase == 1) {
        if (P->fft()) {
            CDV_CUDA(fft_role(P->fftp, P->ga, ROLE_ADJ_TRIAL, c, s), "adjoint trial (FFT)");
            CDV_CUDA(fft_role(P->fftp, P->gf, ROLE_FWD_TRIAL, c, s), "forward trial (FFT)");
        } else if (P->sep()) {
            CDV_CUDA(sep_role(P->sepp, false, ROLE_ADJ_TRIAL, c, s), "adjoint trial (separable)");
            CDV_CUDA(sep_role(P->sepp, true, ROLE_FWD_TRIAL, c, s), "forward trial (separable)");
        } else if (P->tc()) {
            TcArgs F = P->tcf, A = P->tca;
            F.ctx = c;
            A.ctx = c;
            F.role = ROLE_FWD_TRIAL;
            A.role = ROLE_ADJ_TRIAL;
            A.var = (R.o.tikhonov != 0.0 || R.o.armijo != 0.0 || R.o.bb != 0) ? 1 : 0;
            CDV_CUDA(tc_launch(A, P->map_r, s), "adjoint trial (tensor cores)");
            CDV_CUDA(tc_launch(F, P->map_x, s), "forward trial (tensor cores)");
        } else {
            ConvLaunch F{};
            F.g = P->gf;
            F.w = P->H;
            F.batch = 1;
            F.ctx = c;
            ConvLaunch A = F;
            A.g = P->ga;
            A.w = P->Ht;
            F.role = ROLE_FWD_TRIAL;
            A.role = ROLE_ADJ_TRIAL;
            CDV_CUDA(conv_fp32_launch(A, P->ta, s), "adjoint trial");
            CDV_CUDA(conv_fp32_launch(F, P->tf, s), "forward trial");
        }
        CDV_CUDA(decide(0), "decide");
    } else {
        CDV_CUDA(launch_finalize(c, P->nx, s), "finalize");
    }
    return CDV_OK;
}

// Stream form: the prologue, K + max_rejects trial slots (slots after the run has finished return at
// once) and the epilogue.
static cdv_status enqueue_run(cdv_plan* P, const float* Y, float* X, int K, const cdv_iter_opts& o, cudaStream_t s)
{
    RunCtx R{P, Y, X, K, o};
    cdv_status st = run_phase(&R, 0, false, 0, s);
    for (int i = 0; st == CDV_OK && K > 0 && i < K + o.max_rejects; i++) st = run_phase(&R, 1, false, 0, s);
    if (st == CDV_OK) st = run_phase(&R, 2, false, 0, s);
    return st;
}

static cdv_status fill_report(cdv_plan* P, int K, cdv_iter_report* rep, cudaStream_t s)
{
    CDV_CUDA(cudaStreamSynchronize(s), "iterate sync");
    IterState st;
    CDV_CUDA(cudaMemcpy(&st, P->st, sizeof st, cudaMemcpyDeviceToHost), "read state");
    int derr = 0;
    CDV_CUDA(cudaMemcpy(&derr, P->dev_err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
    rep->accepted = st.accepted;
    rep->rejected = st.rejected;
    rep->status = derr ? derr : st.status;
    if (derr) CDV_CUDA(cudaMemset(P->dev_err, 0, sizeof(int)), "clear error word");   // reported here
    rep->trials = st.trials;
    double f0 = 0.0;
    CDV_CUDA(cudaMemcpy(&f0, P->f_hist, sizeof(double), cudaMemcpyDeviceToHost), "read f0");
    rep->f0 = f0;
    rep->f_final = st.f_cur;
    rep->gmac = (double)(1 + st.trials + st.adj_convs) * (double)P->nx * (double)P->nh * 1e-9;
    const int nh = std::min(st.accepted, std::min(K, kHistCap));
    if (rep->f_hist)
        CDV_CUDA(cudaMemcpy(rep->f_hist, P->f_hist, (nh + 1) * sizeof(double), cudaMemcpyDeviceToHost), "read f");
    if (rep->delta_hist && nh > 0)
        CDV_CUDA(cudaMemcpy(rep->delta_hist, P->d_hist, nh * sizeof(double), cudaMemcpyDeviceToHost), "read delta");
    return CDV_OK;
}

cdv_status cdv_iterate(cdv_plan* plan, const float* Y, float* X, int K, const cdv_iter_opts* opts,
                       cdv_iter_report* rep, void* stream)
{
    if (!plan || !Y || !X) return fail(CDV_ERR_INVALID_ARG, "NULL argument");
    if (K < 0) return fail(CDV_ERR_INVALID_ARG, "K = %d", K);
    if (!plan->has_psf) return fail(CDV_ERR_NO_PSF, "no template set");
    cdv_iter_opts o;
    if (opts) o = *opts; else cdv_iter_opts_default(&o);
    if (o.x0_policy < CDV_X0_GIVEN || o.x0_policy > CDV_X0_ZERO) return fail(CDV_ERR_INVALID_ARG, "x0 policy");
    if (!(o.beta > 0.0 && o.beta < 1.0)) return fail(CDV_ERR_INVALID_ARG, "beta = %g", o.beta);
    if (o.max_halvings < 0 || o.max_rejects < 0 || o.max_rejects > 1 << 20)
        return fail(CDV_ERR_INVALID_ARG, "max_halvings/max_rejects");
    if (o.path == CDV_PATH_PERSISTENT)
        return fail(CDV_ERR_UNSUPPORTED, "CDV_PATH_PERSISTENT is the batched solver's path (cdv_batch_iterate)");
    if (o.path < CDV_PATH_AUTO || o.path > CDV_PATH_SMALL) return fail(CDV_ERR_INVALID_ARG, "path = %d", o.path);
    if (!(o.tikhonov >= 0.0 && o.tikhonov < 1e300)) return fail(CDV_ERR_INVALID_ARG, "tikhonov = %g", o.tikhonov);
    if (!(o.armijo >= 0.0 && o.armijo < 1.0)) return fail(CDV_ERR_INVALID_ARG, "armijo = %g", o.armijo);
    if (o.bb != 0 && o.bb != 1) return fail(CDV_ERR_INVALID_ARG, "bb = %d", o.bb);
    const bool plain_rule = o.tikhonov == 0.0 && o.armijo == 0.0 && o.bb == 0;
    const double delta0 = o.delta0 > 0.0 ? o.delta0 : 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    const bool small_ok = plan->mode == CDV_MODE_FP32 && small_supported(plan->m, plan->p);
    if (o.path == CDV_PATH_SMALL && !small_ok)
        return fail(CDV_ERR_UNSUPPORTED, "problem does not fit the single-CTA path (%zu bytes of shared memory)",
                    small_smem_bytes(plan->m, plan->p));
    if (o.path == CDV_PATH_SMALL && !plain_rule)
        return fail(CDV_ERR_UNSUPPORTED, "the single-CTA path runs the plain step rule (tikhonov = armijo = bb = 0)");
    if (!plain_rule && o.path == CDV_PATH_AUTO) o.path = CDV_PATH_GENERAL;
    if (o.path == CDV_PATH_SMALL || (o.path == CDV_PATH_AUTO && small_ok)) {
        SmallRun r{};
        for (int i = 0; i < 3; i++) {
            r.m[i] = plan->m[i];
            r.p[i] = plan->p[i];
        }
        r.y = Y;
        r.x = X;
        r.h = plan->H;
        r.st = plan->st;
        r.f_hist = plan->f_hist;
        r.d_hist = plan->d_hist;
        r.hist_cap = kHistCap;
        r.K = K;
        r.x0_policy = o.x0_policy;
        r.max_halvings = o.max_halvings;
        r.max_rejects = o.max_rejects;
        r.delta0 = delta0;
        r.beta = o.beta;
        r.absum = plan->absum;
        CDV_CUDA(small_iterate(r, s, false), "single-CTA iterate");
        if (rep) return fill_report(plan, K, rep, s);
        return CDV_OK;
    }
    if (o.use_graph) {
        cdv_plan::Key k{Y, X, K, o.x0_policy, o.max_halvings, o.max_rejects, delta0, o.beta, o.tikhonov, o.armijo, o.bb,
                        0};
        const bool same = plan->key_valid && memcmp(&k, &plan->key, sizeof k) == 0;
        if (!same) {
            if (plan->gexec) cudaGraphExecDestroy(plan->gexec);
            if (plan->graph) cudaGraphDestroy(plan->graph);
            plan->gexec = nullptr;
            plan->graph = nullptr;
            plan->key_valid = false;
            // prologue -> WHILE(trial slot) -> epilogue: the device-side decision ends the loop, so no
            // spare slots are launched
            RunCtx R{plan, Y, X, K, o};
            cudaGraph_t gr = nullptr;
            cdv_status st = build_loop_graph(plan->cap, run_phase, &R, &gr);
            if (st != CDV_OK) return st;
            plan->graph = gr;
            CDV_CUDA(cudaGraphInstantiate(&plan->gexec, gr, 0), "instantiate graph");
            plan->key = k;
            plan->key_valid = true;
        }
        CDV_CUDA(cudaGraphLaunch(plan->gexec, s), "graph launch");
    } else {
        cdv_status st = enqueue_run(plan, Y, X, K, o, s);
        if (st != CDV_OK) return st;
    }
    if (rep) return fill_report(plan, K, rep, s);
    return CDV_OK;
}

cdv_status cdv_iterate_host(cdv_plan* plan, const float* Y_host, float* X_host, int K, const cdv_iter_opts* opts,
                            cdv_iter_report* rep, void* stream)
{
    if (!plan || !Y_host || !X_host) return fail(CDV_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    cdv_iter_opts o;
    if (opts) o = *opts; else cdv_iter_opts_default(&o);
    CDV_CUDA(cudaMemcpyAsync(plan->ydev, Y_host, plan->ny * sizeof(float), cudaMemcpyHostToDevice, s), "copy Y in");
    if (o.x0_policy == CDV_X0_GIVEN)
        CDV_CUDA(cudaMemcpyAsync(plan->xdev, X_host, plan->nx * sizeof(float), cudaMemcpyHostToDevice, s), "copy X in");
    cdv_status st = cdv_iterate(plan, plan->ydev, plan->xdev, K, &o, nullptr, stream);
    if (st != CDV_OK) return st;
    CDV_CUDA(cudaMemcpyAsync(X_host, plan->xdev, plan->nx * sizeof(float), cudaMemcpyDeviceToHost, s), "copy X out");
    if (rep) return fill_report(plan, K, rep, s);
    CDV_CUDA(cudaStreamSynchronize(s), "iterate_host sync");
    return CDV_OK;
}

cdv_status cdv_richardson_lucy(cdv_plan* plan, const float* Y, float* X, int K, void* stream)
{
    if (!plan || !Y || !X) return fail(CDV_ERR_INVALID_ARG, "NULL argument");
    if (plan->mode != CDV_MODE_FP32) return fail(CDV_ERR_UNSUPPORTED, "Richardson-Lucy runs in CDV_MODE_FP32 only");
    if (K < 0) return fail(CDV_ERR_INVALID_ARG, "K = %d", K);
    if (!plan->has_psf) return fail(CDV_ERR_NO_PSF, "no template set");
    cudaStream_t s = (cudaStream_t)stream;
    // A^T 1 once
    CDV_CUDA(launch_fill(plan->r0, plan->ny, 1.f, s), "fill");
    cdv_status st = run_conv(plan, false, 1, plan->r0, plan->aux, s);
    if (st != CDV_OK) return st;
    ConvLaunch F{};
    F.g = plan->gf;
    F.w = plan->H;
    F.batch = 1;
    F.ctx = make_ctx(plan, Y, X);
    F.in = X;
    F.out = plan->r0;
    F.y = Y;
    F.role = ROLE_RL_RATIO;
    ConvLaunch A = F;
    A.g = plan->ga;
    A.w = plan->Ht;
    A.in = plan->r0;
    A.out = nullptr;
    A.role = ROLE_RL_UPDATE;
    for (int k = 0; k < K; k++) {
        CDV_CUDA(conv_fp32_launch(F, plan->tf, s), "RL forward");
        CDV_CUDA(conv_fp32_launch(A, plan->ta, s), "RL adjoint");
    }
    return CDV_OK;
}

cdv_status cdv_plan_set_wait_cycles(cdv_plan* plan, long long cycles)
{
    if (!plan) return fail(CDV_ERR_INVALID_ARG, "plan is NULL");
    if (cycles < 0) return fail(CDV_ERR_INVALID_ARG, "cycles = %lld", cycles);
    const long long c = cycles == 0 ? kTcWaitCycles : cycles;
    plan->tcf.wait_cycles = c;
    plan->tca.wait_cycles = c;
    plan->key_valid = false;               // a captured graph holds the old launch parameters
    return CDV_OK;
}

cdv_status cdv_plan_sync_status(cdv_plan* plan, void* stream)
{
    if (!plan) return fail(CDV_ERR_INVALID_ARG, "plan is NULL");
    CDV_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "sync");
    CDV_CUDA(cudaGetLastError(), "pending error");
    int derr = 0;
    CDV_CUDA(cudaMemcpy(&derr, plan->dev_err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
    if (derr) {
        CDV_CUDA(cudaMemset(plan->dev_err, 0, sizeof(int)), "clear error word");
        return fail((cdv_status)derr, "device-side error recorded by a kernel");
    }
    return CDV_OK;
}

}  // extern "C"

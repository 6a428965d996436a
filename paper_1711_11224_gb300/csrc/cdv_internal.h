// Internal declarations shared by the CUDA translation units of libcdv.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/cdv.h"

namespace cdv {

// What a convolution launch computes around the sum
//   out[s] = sum_j w[j] * in[s + o - j]
// (forward: in = X, o = 0, w = H; adjoint: in = R, o = 2p, w = H~).
enum Role : int {
    ROLE_PLAIN = 0,      // out = sum
    ROLE_FWD_INIT = 1,   // r[cur] = A x[cur] - y, FP64 partials of ||r||^2
    ROLE_FWD_TRIAL = 2,  // r[cur^1] = A x[cur^1] - y, FP64 partials of ||r||^2
    ROLE_ADJ_TRIAL = 3,  // g = A^T r[cur] (unless reusing g), x[cur^1] = max(x[cur] - delta g, 0),
                         // FP64 partials of ||x[cur^1] - x[cur]||^2
    ROLE_RL_RATIO = 4,   // out = y / sum (0 where sum == 0)           (Richardson-Lucy)
    ROLE_RL_UPDATE = 5,  // x = x * sum / norm (0 where norm == 0)     (Richardson-Lucy)
};

// Device-resident scalars of the projected-gradient iteration (FP64).
struct IterState {
    double f_cur;        // f(x_k)
    double f_trial;      // f of the last trial
    double delta;        // step length of the next trial
    double delta0, beta;
    double moved;        // ||x_trial - x_k||^2 of the last trial
    int accepted, rejected, halvings, max_halvings;
    int max_rejects, K, cur, need_grad;
    int done, status, trials, hist_cap;
    int adj_convs, pad_;
    double lambda;       // Tikhonov weight: f = 1/2 ||A x - y||^2 + lambda/2 ||x||^2
    double sigma;        // Armijo factor: accept iff f_t < f_k + sigma <grad f(x_k), x_t - x_k>
    double sy;           // <x_k - x_{k-1}, grad f(x_k) - grad f(x_{k-1})> of the current step (bb)
    double ss_last;      // ||x_k - x_{k-1}||^2 of the last accepted step (bb)
    int bb, pad2_;       // bb: Barzilai-Borwein first trials, lagged by one step
};

struct IterCtx {
    float* x[2];         // x[0]: caller's X, x[1]: workspace
    float* r[2];         // residual buffers (size of Y)
    float* g;            // gradient A^T r (size of X)
    const float* y;      // observation
    const float* aux;    // Richardson-Lucy: A^T 1
    double* part_f;      // per-CTA partials of ||r||^2
    double* part_m;      // per-CTA partials of ||x_trial - x||^2
    double* part_a;      // per-CTA partials of <grad f(x_k), x_trial - x_k> (used when sigma != 0)
    double* part_x;      // per-CTA partials of ||x_trial||^2 (used when lambda != 0)
    double* part_sy;     // per-CTA partials of <x_k - x_{k-1}, grad f(x_k) - grad f(x_{k-1})> (bb)
    IterState* st;
    double* f_hist;      // hist_cap + 1 entries
    double* d_hist;      // hist_cap entries
};

// Geometry of one convolution, always 3-D (leading axes of size 1 for n < 3).
struct ConvGeom {
    int64_t a1, a2, a3;  // input dims
    int64_t b1, b2, b3;  // output dims
    int o1, o2, o3;      // offsets (0 forward, 2p adjoint)
    int q1, q2, q3;      // template dims
};

struct ConvLaunch {
    ConvGeom g;
    const float* in;
    float* out;
    const float* w;      // q1*q2*q3 weights in C-order
    const float* y;      // ROLE_RL_RATIO: observation
    int role;
    int batch;
    int64_t in_bstride, out_bstride;
    IterCtx ctx;
};

// Tile shape of the FP32 engine chosen for one geometry.
struct ConvTile {
    int ntx, nty;        // threads along axis 3 and axis 2
    int tiles1, tiles2, tiles3;
    int grid;            // CTAs per volume
    size_t smem;         // dynamic shared memory bytes
};

// One volume of a batched launch of the FP32 engine.
struct ConvBatchVol {
    ConvLaunch L;
    int ntx, nty, tiles2, tiles3;
    size_t smem;
};

// FP32 direct-convolution engine (CUDA cores).
bool conv_fp32_supported(int q3);
ConvTile conv_fp32_tile(const ConvGeom& g);
cudaError_t conv_fp32_launch(const ConvLaunch& L, const ConvTile& t, cudaStream_t s);
cudaError_t conv_fp32_prepare(int q3);   // once per process and width, outside stream capture
cudaError_t grad_psf_prepare();

// Per-Q3 launchers (one translation unit per group of template widths).
template <int Q3>
cudaError_t conv_fp32_launch_q(const ConvLaunch& L, const ConvTile& t, cudaStream_t s);
template <int Q3>
cudaError_t conv_fp32_batch_launch_q(const ConvBatchVol* vols, const int2* items, int nitems, size_t smem,
                                     cudaStream_t s);
// Batched launch over a work list (volume, tile) of volumes sharing template width q3; nitems == 0
// prepares the kernel (outside stream capture).
cudaError_t conv_fp32_batch_launch(int q3, const ConvBatchVol* vols, const int2* items, int nitems, size_t smem,
                                   cudaStream_t s);
ConvTile conv_fp32_tile_shape(const ConvGeom& g, int nty);

// Iteration kernels (iterate.cu).
cudaError_t launch_x0(int policy, float* x, const float* y, int64_t m1, int64_t m2, int64_t m3,
                      int p1, int p2, int p3, cudaStream_t s);
cudaError_t launch_state_init(IterState* st, double delta0, const double* absum, double beta, int max_halvings,
                              int max_rejects, int K, int hist_cap, double lambda, double sigma, int bb,
                              cudaStream_t s);
cudaError_t launch_sumsq(const float* x, int64_t n, double* out, cudaStream_t s);
cudaError_t launch_decide(const IterCtx& c, int nparts_f, int nparts_m, int init, cudaStream_t s);
cudaError_t launch_decide_loop(const IterCtx& c, int nparts_f, int nparts_m, int init, unsigned long long handle,
                               int max_trials, cudaStream_t s);
cudaError_t launch_finalize(const IterCtx& c, int64_t nx, cudaStream_t s);

// Batched iteration: per-volume context read by the batched kernels.
struct BatchVolCtx {
    IterCtx c;
    int64_t m1, m2, m3;
    int p1, p2, p3;
    int nparts_f, nparts_m;
    const double* absum;
};
cudaError_t launch_batch_x0(const BatchVolCtx* v, int count, int policy, cudaStream_t s);
cudaError_t launch_batch_state_init(const BatchVolCtx* v, int count, double delta0, double beta, int max_halvings,
                                    int max_rejects, int K, int hist_cap, cudaStream_t s);
cudaError_t launch_batch_decide(const BatchVolCtx* v, int count, int init, cudaStream_t s);
cudaError_t launch_batch_finalize(const BatchVolCtx* v, int count, cudaStream_t s);
cudaError_t launch_batch_loop_cond(const BatchVolCtx* v, int count, unsigned long long handle, int max_trials,
                                   cudaStream_t s);

// Persistent batched solver (conv_fp32_persist.cu): every volume's whole run in one launch.
struct BatchPersist {
    const ConvBatchVol* fi;      // per volume: initial forward, forward trial, adjoint trial
    const ConvBatchVol* ft;
    const ConvBatchVol* at;
    const BatchVolCtx* ctx;
    const int* order;            // volumes in scan order (most work first)
    const int2* ntiles;          // per scan position: forward tiles (x), adjoint tiles (y)
    unsigned long long* word;    // per scan position: phase (high 32 bits) and next tile (low 32 bits), zero at start
    int* tiles_done;             // per volume: tiles of the current phase completed, zero at start
    int* vols_done;              // volumes retired, zero at start
    int* err;                    // CDV_ERR_TIMEOUT when a CTA found no tile for wait_cycles
    int count, max_trials;
    long long wait_cycles;
};
cudaError_t conv_fp32_persist_prepare();                 // once per process, outside stream capture
int conv_fp32_persist_grid(size_t smem);                 // resident CTAs of the kernel (SMs x CTAs per SM)
cudaError_t conv_fp32_persist_launch(const BatchPersist& P, int grid, size_t smem, cudaStream_t s);

// CUDA graph "prologue -> WHILE(body) -> epilogue": `phase` enqueues phase 0 (prologue), 1 (one trial
// slot; its last kernel sets the loop condition through the handle) or 2 (epilogue) on a stream.
typedef cdv_status (*PhaseFn)(void* ctx, int phase, bool loop, unsigned long long handle, cudaStream_t s);
cdv_status build_loop_graph(cudaStream_t cap, PhaseFn phase, void* ctx, cudaGraph_t* out);

// Template preparation (psf.cu).
cudaError_t launch_flip(const float* h, float* ht, int q1, int q2, int q3, cudaStream_t s);
cudaError_t launch_abs_sum(const float* h, int64_t n, double* out, cudaStream_t s);

// Template gradient (grad_psf.cu).
struct GradPsfPlan {
    int64_t m1, m2, m3;
    int q1, q2, q3;
    int batch;
    int chunks;          // slabs of axis 1 reduced separately
};
// Dynamic shared memory of one grad_psf_kernel block for this plan (0: more than 1024 threads);
// launches above kGradPsfMaxSmem fail with cudaErrorInvalidConfiguration.
constexpr size_t kGradPsfMaxSmem = 227 * 1024;
size_t grad_psf_smem_bytes(const GradPsfPlan& g);
int grad_psf_chunks(const GradPsfPlan& g);      // chunks for a plan (after grad_psf_prepare)
size_t grad_psf_partials(const GradPsfPlan& g);
cudaError_t launch_grad_psf(const GradPsfPlan& g, const float* X, const float* dY, double* partial,
                            float* dH, cudaStream_t s);

// Whole-run kernel for problems that fit in one SM's shared memory (small.cu).
struct SmallRun {
    int64_t m[3];
    int p[3];
    const float* y;
    float* x;
    const float* h;
    IterState* st;
    double* f_hist;
    double* d_hist;
    int hist_cap, K, x0_policy, max_halvings, max_rejects;
    double delta0, beta;
    const double* absum;
};
bool small_supported(const int64_t* m, const int* p);
size_t small_smem_bytes(const int64_t* m, const int* p);
cudaError_t small_iterate(const SmallRun& r, cudaStream_t s, bool prepare);

// Tensor-core engine (conv_tc.cu).  One launch = one convolution over the
// whole volume; the input is read through TMA from BF16/TF32 shadow copies
// in a padded layout, the FP32 output and the shadows of the output are
// written by the epilogue.
struct TcArgs {
    ConvGeom g;
    int role, kind, nprec;
    int e;               // window pad: K index 0 is input column S3 + o3 - (q3-1) - e
    int K;               // window length (elements), multiple of 16
    int kchunks;         // 16-byte chunks along K
    int W;               // output columns per plane of a tile (8 or 16)
    int P;               // output planes per CTA (P x W = 128 accumulator columns per M tile)
    int MT;              // 128-row M tiles per CTA
    int rows;            // staged input rows (>= 128*MT + q2 - 1), two TMA boxes of rows/2
    int na, ns;          // input-plane buffers, template-tile stages
    int tiles1, tiles2, tiles3;
    int ntiles;          // output tiles (tiles1 x tiles2 x tiles3)
    int grid;            // persistent CTAs (at most one per SM), each walking tiles blockIdx.x + k * grid
    int var;             // 1: the instantiation with the iteration's step-rule variants (per launch)
    unsigned tmem_cols;
    int64_t sh_pitch;    // row pitch of the output shadows
    float* out;          // ROLE_PLAIN output
    const void* bt[2];   // Toeplitz tiles [part][j2][K chunk][j1*16 + n][16 bytes]
    void* sh_out_hi[2];
    void* sh_out_lo[2];
    int* err;            // device error word
    long long wait_cycles;   // budget of each barrier wait in the work loops (clock64 cycles)
    // narrow form (conv_tc4.cuh): 4 output columns per tile, 32 output-plane slots
    int w4;              // 1: this direction runs the narrow kernel
    int pc;              // output planes per tile (a multiple of 32)
    int kc;              // 16-byte chunks of the window of 4 + q3 - 1 columns
    int steps;           // MMA K steps per input plane: ceil(q2 * kc / 2)
    int spst;            // K steps per template stage
    int nst;             // template stages per input plane
    int64_t sh_pitch1;   // row pitch of the output shadows shifted by 4 columns
    // forward only: M runs over (column group, row) of the groups of copy 0, then those of copy 1, rows
    // padded to lp (a multiple of 32, >= b2); each window chunk is staged in 32-row boxes, each box from
    // the copy its group belongs to
    int flat;
    int lp;
    int fboxes;          // 32-row boxes per window chunk of one staged input plane (one part)
    int ngrp[2];         // column groups per shadow copy
    int gfirst[2];       // first column group of each copy
    int nblk;            // 256-row M blocks over the groups of both copies
    // per-CTA tile lists: CTA b walks tlist[toff[b] .. toff[b + 1]), each tile {S1, s1_end, combo, 0}:
    // output planes [S1, s1_end) (S1 a multiple of 32) of M block `combo` (flat: index over the copies'
    // blocks; else row block * column groups + column group)
    const int4* tlist;
    const int* toff;
    void* sh_out_hi1[2];
    void* sh_out_lo1[2];
    IterCtx ctx;
};
constexpr long long kTcWaitCycles = 1000000000ll;   // default budget, about 0.5 s
size_t tc_smem_bytes(const TcArgs& t);
cudaError_t tc_prepare(int kind);
cudaError_t tc_launch(const TcArgs& t, const struct CUtensorMap_st* maps, cudaStream_t s);
cudaError_t tc_build_btiles(const float* w, int q1, int q2, int q3, int D, int K, int W, int kind, void* hi,
                            void* lo, cudaStream_t s);
cudaError_t tc_shadow(const float* src, int64_t a1a2, int64_t a3, int64_t pitch, int kind, void* hi, void* lo,
                      cudaStream_t s);
// Narrow form (conv_tc4.cu): shared-memory bytes, launch (maps: copy 0 hi0 lo0 hi1 lo1, then copy 1),
// template stages ([part][stage][version][group][chunk][8 rows][16 B]), the shifted shadow copy
// (column c at c + 4 of a row of pitch1; columns 0-3 are never written and must hold zeros).
size_t tc4_smem_bytes(const TcArgs& t);
size_t tc4_btiles_bytes(const TcArgs& t);
cudaError_t tc4_prepare(int kind);
cudaError_t tc4_launch(const TcArgs& t, const struct CUtensorMap_st* maps, cudaStream_t s);
cudaError_t tc4_build_btiles(const TcArgs& t, const float* w, void* hi, void* lo, cudaStream_t s);
cudaError_t tc4_shadow1(const float* src, int64_t a1a2, int64_t a3, int64_t pitch1, int kind, void* hi, void* lo,
                        cudaStream_t s);
// Balanced tile lists for the narrow kernel (host): fills the tile lists and the grid, returns the
// modelled makespan in cycles; tc4_executed_macs counts the MMAs of those lists.
double tc4_partition(TcArgs& t, int nsm, int pc, std::vector<int4>& list, std::vector<int>& off);
void tc4_window_extent(const TcArgs& t, int64_t need[2]);
double tc4_executed_macs(const TcArgs& t, const std::vector<int4>& list);

// FFT comparator (fft.cu): cuFFT plans over the zero-padded grid of N_i >= m_i + 2p_i samples.
struct FftPlan {
    int64_t N[3] = {1, 1, 1};
    int64_t nreal = 0, ncplx = 0;
    int r2c = 0, c2r = 0;     // cufftHandle
    bool have_plans = false;
    float* real = nullptr;    // nreal floats
    void* spec = nullptr;     // ncplx cufftComplex: the transform of the current input
    void* hspec = nullptr;    // ncplx cufftComplex: transform of the zero-padded template / prod(N)
};
int fft_epilogue_blocks();
cudaError_t fft_setup(FftPlan& F, const ConvGeom& gf, void* (*alloc)(void* owner, size_t bytes), void* owner);
void fft_release(FftPlan& F);
cudaError_t fft_set_psf(FftPlan& F, const float* H, int q1, int q2, int q3, cudaStream_t s);
cudaError_t fft_conv(FftPlan& F, const ConvGeom& g, bool fwd, const float* in, float* out, cudaStream_t s);
cudaError_t fft_role(FftPlan& F, const ConvGeom& g, int role, const IterCtx& c, cudaStream_t s);

// Unsigned 32-bit division by a divisor fixed at plan time, as a multiply-high and two shifts
// (Granlund and Montgomery, "Division by invariant integers using multiplication", 1994).
struct FastDiv {
    uint32_t m;
    int s1, s2;
};
FastDiv make_fastdiv(uint32_t d);

// Separable-template engine (sep.cu).  One 1-D pass over a volume viewed as (outer, kin, inner):
//   out[u, s, i] = sum_{j < q} w[j] in[u, s + o - j, i]   (in = 0 outside [0, kin))
struct SepPass {
    const float* in;     // null on the first pass of a role launch: chosen from the iteration state
    float* out;          // null on the last pass of a role launch: the epilogue's buffers
    const float* w;      // q taps
    int64_t outer, kin, kout, inner;
    int q, o;
    int first, last;
    int role;
    int seg, rb;         // rows kernel (inner == 1): outputs per segment (multiple of 7), rows per task
    FastDiv dspan, dcpr, dseg;   // rows kernel: division by seg + q - 1, seg / 7 and seg
    int64_t strip;       // cols kernel: outputs per warp task (multiple of 8)
    IterCtx c;
};
struct SepPlan {
    float* hf = nullptr;     // factors h_1 | h_2 | h_3 (q1 + q2 + q3 floats)
    float* hb = nullptr;     // the same, each reversed (the factors of H~)
    float* tA = nullptr;     // intermediates, m1 x (m2 + 2p2) x (m3 + 2p3) floats each
    float* tB = nullptr;
    SepPass fwd[3], adj[3];
};
int sep_blocks();
bool sep_supported(const int q[3]);
cudaError_t sep_setup(SepPlan& S, const int64_t m[3], const int p[3], void* (*alloc)(void* owner, size_t bytes),
                      void* owner);
// h[a]: device pointer to q[a] floats (null: the axis has q[a] == 1 and factor 1); H receives the
// dense outer product.
cudaError_t sep_set_factors(SepPlan& S, const float* const h[3], const int q[3], float* H, cudaStream_t s);
cudaError_t sep_conv(const SepPlan& S, bool fwd, const float* in, float* out, cudaStream_t s);
cudaError_t sep_role(const SepPlan& S, bool fwd, int role, const IterCtx& c, cudaStream_t s);
double sep_pass_macs(const SepPlan& S, bool fwd);
template <int Q, bool EPI>
cudaError_t sep_launch_q(const SepPass& P, int blocks, cudaStream_t s);

// Message returned by cdv_last_error() on this host thread (capi.cu).
void set_last_error(const char* msg);

// Elementwise helpers (iterate.cu).
cudaError_t launch_fill(float* x, int64_t n, float v, cudaStream_t s);

}  // namespace cdv

// Step rule of the iteration (Step 2 and its options), shared by the per-launch decision kernels
// (iterate.cu) and the persistent batched solver (conv_fp32_persist.cu).
#pragma once

#include <math.h>

#include "cdv_internal.h"

namespace cdv {

// Deterministic FP64 sum of n partials by one block: strided per-thread sums
// in index order, then a fixed shared-memory tree.
static __device__ __forceinline__ double block_reduce_fixed(const double* a, int n, double* sh)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += a[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double t = sh[0];
    __syncthreads();
    return t;
}

// The same sum, in the same order as block_reduce_fixed with 512 threads, by a block of 256 (thread t
// forms the strided sums of t and t + 256; sh holds 512 values).
static __device__ __forceinline__ double block_reduce_fixed512(const double* a, int n, double* sh)
{
    const int t = threadIdx.x;
    double s0 = 0.0, s1 = 0.0;
    for (int i = t; i < n; i += 512) s0 += a[i];
    for (int i = t + 256; i < n; i += 512) s1 += a[i];
    sh[t] = s0;
    sh[t + 256] = s1;
    __syncthreads();
    for (int w = 256; w > 0; w >>= 1) {
        if (t < w) sh[t] += sh[t + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

struct ReduceBlock {
    __device__ double operator()(const double* a, int n, double* sh) const { return block_reduce_fixed(a, n, sh); }
};
struct Reduce512On256 {
    __device__ double operator()(const double* a, int n, double* sh) const { return block_reduce_fixed512(a, n, sh); }
};

// One decision of the step rule for the run in c (init: the initial forward's f(x_0)); thread 0
// updates the state, every thread of the block takes part in the reductions.
template <class Reduce>
static __device__ void decide_body_r(const IterCtx& c, int nf, int nm, int init, double* sh, Reduce red)
{
    IterState* st = c.st;
    if (st->done) return;
    const double lambda = st->lambda, sigma = st->sigma;
    double F = 0.5 * red(c.part_f, nf, sh);
    const double M = init ? 0.0 : red(c.part_m, nm, sh);
    if (lambda != 0.0) F += 0.5 * lambda * red(c.part_x, init ? 1 : nm, sh);
    const double D = (sigma != 0.0 && !init) ? red(c.part_a, nm, sh) : 0.0;
    // the first trial of a step (a fresh gradient) also brought <x_k - x_{k-1}, grad f(x_k) - grad f(x_{k-1})>
    const bool new_sy = st->bb && !init && st->need_grad && st->accepted >= 1;
    const double SY = new_sy ? red(c.part_sy, nm, sh) : 0.0;
    if (threadIdx.x != 0) return;
    if (new_sy) st->sy = SY;
    if (init) {
        st->f_cur = F;
        c.f_hist[0] = F;
        st->need_grad = 1;
        if (!isfinite(F)) {
            st->status = CDV_ERR_NONFINITE;
            st->done = 1;
        } else if (st->K <= 0) {
            st->done = 1;
        }
        return;
    }
    st->trials += 1;
    if (st->need_grad) st->adj_convs += 1;
    st->f_trial = F;
    st->moved = M;
    if (M == 0.0) {                       // x_t == x_k: stationary point, the run has converged
        st->status = CDV_ERR_NOT_DESCENDING;
        st->done = 1;
        return;
    }
    if (!isfinite(F)) {
        st->status = CDV_ERR_NONFINITE;
        st->done = 1;
        return;
    }
    if (F < st->f_cur + sigma * D) {      // f(x_{k+1}) < f(x_k) (+ sigma <grad f, x_{k+1} - x_k>): accept
        const int a = st->accepted;
        if (a < st->hist_cap) {
            c.d_hist[a] = st->delta;
            c.f_hist[a + 1] = F;
        }
        st->accepted = a + 1;
        st->cur ^= 1;
        st->f_cur = F;
        st->halvings = 0;
        if (st->bb) {                     // next step: <s,s>/<s,v> of (x_k - x_{k-1}, grad f(x_k) - grad f(x_{k-1}))
            double d = st->delta0;
            if (a >= 1) {
                const double dmax = st->delta0 * 1048576.0;
                d = st->sy > 0.0 ? st->ss_last / st->sy : dmax;
                d = fmin(fmax(d, st->delta0), dmax);
            }
            st->ss_last = M;              // ||x_{k+1} - x_k||^2 for the step after
            st->delta = d;
        } else {
            st->delta = st->delta0;
        }
        st->need_grad = 1;
        if (st->accepted >= st->K) st->done = 1;
    } else {                              // reject: shorten the step, keep x_k and g_k
        st->rejected += 1;
        st->halvings += 1;
        st->need_grad = 0;
        if (st->halvings > st->max_halvings || st->rejected > st->max_rejects) {
            st->status = CDV_ERR_NOT_DESCENDING;
            st->done = 1;
        } else {
            st->delta *= st->beta;
        }
    }
}

static __device__ __forceinline__ void decide_body(const IterCtx& c, int nf, int nm, int init, double* sh)
{
    decide_body_r(c, nf, nm, init, sh, ReduceBlock{});
}

}  // namespace cdv

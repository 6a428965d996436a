// Device-side control of the projected-gradient iteration (Steps 1-3 of the
// 2-D application, any n) and its elementwise helpers.
//
// One step of the run is a fixed three-launch "trial slot":
//   1. adjoint trial  g = A^T r_k (skipped after a rejected trial, g reused),
//                     x_t = max(x_k - delta (g + lambda x_k), 0), partials of
//                     ||x_t - x_k||^2 (and, when used, of <g + lambda x_k, x_t - x_k>
//                     and ||x_t||^2)
//   2. forward trial  r_t = A x_t - y, partials of ||r_t||^2
//   3. decide         f_t = 1/2 ||r_t||^2 + lambda/2 ||x_t||^2 (FP64, fixed-order
//                     reductions); accept if f_t < f_k + sigma <grad f(x_k), x_t - x_k>
//                     (lambda = sigma = 0: the decrease rule of Step 2),
//                     else delta <- beta * delta and retry from x_k.
// All decisions live in IterState on the device, so the slots of a whole run
// can be captured in one CUDA graph and replayed without host round trips.
// Slots after the run has finished return at once.
#include <math.h>

#include <algorithm>

#include "cdv_internal.h"
#include "decide.cuh"

namespace cdv {

__global__ void x0_kernel(int policy, float* x, const float* y, int64_t m1, int64_t m2, int64_t m3, int p1,
                          int p2, int p3)
{
    const int64_t n = m1 * m2 * m3;
    const int64_t n2 = m2 + 2 * p2, n3 = m3 + 2 * p3;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (policy == CDV_X0_ZERO) {
            x[i] = 0.f;
        } else {
            const int64_t k3 = i % m3, k2 = (i / m3) % m2, k1 = i / (m2 * m3);
            const float v = y[((k1 + p1) * n2 + (k2 + p2)) * n3 + (k3 + p3)];
            x[i] = v > 0.f ? v : 0.f;
        }
    }
}

cudaError_t launch_x0(int policy, float* x, const float* y, int64_t m1, int64_t m2, int64_t m3, int p1, int p2,
                      int p3, cudaStream_t s)
{
    if (policy == CDV_X0_GIVEN) return cudaSuccess;
    const int64_t n = m1 * m2 * m3;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    x0_kernel<<<blocks, 256, 0, s>>>(policy, x, y, m1, m2, m3, p1, p2, p3);
    return cudaGetLastError();
}

__device__ void state_init_kernel_body(IterState* st, double delta0, const double* absum, double beta,
                                       int max_halvings, int max_rejects, int K, int hist_cap, double lambda,
                                       double sigma, int bb)
{
    if (!(delta0 > 0.0)) {                // default step 1/L, L = (sum |h|)^2 + lambda >= ||A||_2^2 + lambda
        const double a = *absum;
        delta0 = 1.0 / (a * a + lambda);
    }
    st->f_cur = 0.0;
    st->f_trial = 0.0;
    st->delta = delta0;
    st->delta0 = delta0;
    st->beta = beta;
    st->moved = 0.0;
    st->accepted = 0;
    st->rejected = 0;
    st->halvings = 0;
    st->max_halvings = max_halvings;
    st->max_rejects = max_rejects;
    st->K = K;
    st->cur = 0;
    st->need_grad = 1;
    st->done = 0;
    st->status = CDV_OK;
    st->trials = 0;
    st->hist_cap = hist_cap;
    st->adj_convs = 0;
    st->pad_ = 0;
    st->lambda = lambda;
    st->sigma = sigma;
    st->sy = 0.0;
    st->ss_last = 0.0;
    st->bb = bb;
    st->pad2_ = 0;
}

__global__ void state_init_kernel(IterState* st, double delta0, const double* absum, double beta, int max_halvings,
                                  int max_rejects, int K, int hist_cap, double lambda, double sigma, int bb)
{
    state_init_kernel_body(st, delta0, absum, beta, max_halvings, max_rejects, K, hist_cap, lambda, sigma, bb);
}

cudaError_t launch_state_init(IterState* st, double delta0, const double* absum, double beta, int max_halvings,
                              int max_rejects, int K, int hist_cap, double lambda, double sigma, int bb,
                              cudaStream_t s)
{
    state_init_kernel<<<1, 1, 0, s>>>(st, delta0, absum, beta, max_halvings, max_rejects, K, hist_cap, lambda, sigma,
                                      bb);
    return cudaGetLastError();
}

// ||x||^2 of the initial iterate in FP64, one block, fixed order (the Tikhonov part of f(x_0)).
__global__ void __launch_bounds__(512) sumsq_kernel(const float* x, int64_t n, double* out)
{
    __shared__ double sh[512];
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v += (double)x[i] * (double)x[i];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

cudaError_t launch_sumsq(const float* x, int64_t n, double* out, cudaStream_t s)
{
    sumsq_kernel<<<1, 512, 0, s>>>(x, n, out);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(512) decide_kernel(IterCtx c, int nf, int nm, int init)
{
    __shared__ double sh[512];
    decide_body(c, nf, nm, init, sh);
}

// Decision inside a CUDA-graph WHILE loop: after the step rule, the loop continues while the run is
// not done; max_trials is a hard cap (K + max_rejects + 1) that always ends the loop.
__global__ void __launch_bounds__(512) decide_loop_kernel(IterCtx c, int nf, int nm, int init,
                                                          cudaGraphConditionalHandle h, int max_trials)
{
    __shared__ double sh[512];
    decide_body(c, nf, nm, init, sh);
    if (threadIdx.x == 0) {
        const IterState* st = c.st;
        cudaGraphSetConditional(h, (st->done || st->trials >= max_trials) ? 0u : 1u);
    }
}

cudaError_t launch_decide_loop(const IterCtx& c, int nparts_f, int nparts_m, int init, unsigned long long handle,
                               int max_trials, cudaStream_t s)
{
    decide_loop_kernel<<<1, 512, 0, s>>>(c, nparts_f, nparts_m, init, (cudaGraphConditionalHandle)handle, max_trials);
    return cudaGetLastError();
}

cudaError_t launch_decide(const IterCtx& c, int nparts_f, int nparts_m, int init, cudaStream_t s)
{
    decide_kernel<<<1, 512, 0, s>>>(c, nparts_f, nparts_m, init);
    return cudaGetLastError();
}

__global__ void finalize_kernel(IterCtx c, int64_t nx)
{
    if (c.st->cur == 0) return;
    const float* src = c.x[1];
    float* dst = c.x[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nx; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

cudaError_t launch_finalize(const IterCtx& c, int64_t nx, cudaStream_t s)
{
    const int blocks = (int)std::min<int64_t>((nx + 255) / 256, 152 * 8);
    finalize_kernel<<<blocks, 256, 0, s>>>(c, nx);
    return cudaGetLastError();
}

__global__ void fill_kernel(float* x, int64_t n, float v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

cudaError_t launch_fill(float* x, int64_t n, float v, cudaStream_t s)
{
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    fill_kernel<<<blocks, 256, 0, s>>>(x, n, v);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- batched forms (one volume per block row)

__global__ void batch_x0_kernel(const BatchVolCtx* v, int policy)
{
    const BatchVolCtx& b = v[blockIdx.y];
    if (policy == CDV_X0_GIVEN) return;
    const int64_t n = b.m1 * b.m2 * b.m3;
    const int64_t n2 = b.m2 + 2 * b.p2, n3 = b.m3 + 2 * b.p3;
    float* x = b.c.x[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (policy == CDV_X0_ZERO) {
            x[i] = 0.f;
        } else {
            const int64_t k3 = i % b.m3, k2 = (i / b.m3) % b.m2, k1 = i / (b.m2 * b.m3);
            const float y = b.c.y[((k1 + b.p1) * n2 + (k2 + b.p2)) * n3 + (k3 + b.p3)];
            x[i] = y > 0.f ? y : 0.f;
        }
    }
}

__global__ void batch_state_init_kernel(const BatchVolCtx* v, int count, double delta0, double beta, int max_halvings,
                                        int max_rejects, int K, int hist_cap)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    state_init_kernel_body(v[i].c.st, delta0, v[i].absum, beta, max_halvings, max_rejects, K, hist_cap, 0.0, 0.0, 0);
}

__global__ void __launch_bounds__(512) batch_decide_kernel(const BatchVolCtx* v, int init)
{
    __shared__ double sh[512];
    const BatchVolCtx& b = v[blockIdx.x];
    decide_body(b.c, b.nparts_f, b.nparts_m, init, sh);
}

__global__ void batch_finalize_kernel(const BatchVolCtx* v)
{
    const BatchVolCtx& b = v[blockIdx.y];
    if (b.c.st->cur == 0) return;
    const int64_t n = b.m1 * b.m2 * b.m3;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b.c.x[0][i] = b.c.x[1][i];
}

// Loop condition of the batched WHILE graph: continue while any volume is still running.
__global__ void batch_loop_cond_kernel(const BatchVolCtx* v, int count, cudaGraphConditionalHandle h, int max_trials)
{
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const IterState* st = v[i].c.st;
        if (!st->done && st->trials < max_trials) atomicOr(&any, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

cudaError_t launch_batch_loop_cond(const BatchVolCtx* v, int count, unsigned long long handle, int max_trials,
                                   cudaStream_t s)
{
    batch_loop_cond_kernel<<<1, 256, 0, s>>>(v, count, (cudaGraphConditionalHandle)handle, max_trials);
    return cudaGetLastError();
}

cudaError_t launch_batch_x0(const BatchVolCtx* v, int count, int policy, cudaStream_t s)
{
    if (policy == CDV_X0_GIVEN) return cudaSuccess;
    batch_x0_kernel<<<dim3(64, count), 256, 0, s>>>(v, policy);
    return cudaGetLastError();
}

cudaError_t launch_batch_state_init(const BatchVolCtx* v, int count, double delta0, double beta, int max_halvings,
                                    int max_rejects, int K, int hist_cap, cudaStream_t s)
{
    batch_state_init_kernel<<<(count + 127) / 128, 128, 0, s>>>(v, count, delta0, beta, max_halvings, max_rejects, K,
                                                                hist_cap);
    return cudaGetLastError();
}

cudaError_t launch_batch_decide(const BatchVolCtx* v, int count, int init, cudaStream_t s)
{
    batch_decide_kernel<<<count, 512, 0, s>>>(v, init);
    return cudaGetLastError();
}

cudaError_t launch_batch_finalize(const BatchVolCtx* v, int count, cudaStream_t s)
{
    batch_finalize_kernel<<<dim3(64, count), 256, 0, s>>>(v);
    return cudaGetLastError();
}

}  // namespace cdv

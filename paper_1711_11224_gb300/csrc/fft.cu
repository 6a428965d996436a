// FFT comparator (CDV_MODE_FFT): the forward and adjoint operators through cuFFT, the approach the
// paper's introduction contrasts with direct convolution.  Not the paper's method; it runs the same
// iteration (same state, decisions and reports) so the two can be set side by side.
//
// Both operators are linear convolutions embedded in one zero-padded periodic grid of N_i >= m_i +
// 2p_i samples per axis (N_i the smallest 2^a 3^b 5^c 7^d at or above it):
//   forward  Y = X (*) H:   FFT(pad X) * FFT(pad H), inverse, keep [0, m + 2p)   (no wrap-around: the
//            full output has m + 2p samples per axis)
//   adjoint  g(k) = sum_j h(j) r(k + j):  FFT(pad R) * conj(FFT(pad H)), inverse, keep [0, m)   (for
//            k < m and j <= 2p, k + j < m + 2p <= N; negative shifts meet the zero tail of pad H)
// The template spectrum carries the 1/prod(N) of the unnormalised inverse transform.
// In the iteration the pad kernel picks the input buffer and the crop kernel the output buffer from the
// device state (as the direct kernels do), and the crop kernels fuse the residual, the projected
// update and the FP64 block partials of the direct engines' epilogues.
#include <cufft.h>

#include <algorithm>

#include "cdv_internal.h"

namespace cdv {

namespace {

constexpr int kEpiBlocks = 152 * 4;
constexpr int kEpiThreads = 256;

int64_t good_size(int64_t n)
{
    for (int64_t v = std::max<int64_t>(n, 1);; v++) {
        int64_t r = v;
        for (int f : {2, 3, 5, 7})
            while (r % f == 0) r /= f;
        if (r == 1) return v;
    }
}

__device__ __forceinline__ double block_sum(double v, double* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += sh[i];
    return t;
}

// Zero-padded copy of a (d1, d2, d3) volume into the (N1, N2, N3) real grid.  `src` null: the input
// is chosen from the iteration state (sel: 0 x[cur], 1 x[cur ^ 1], 2 r[cur]).
__global__ void fft_pad_kernel(const float* src, int sel, IterCtx c, int64_t d1, int64_t d2, int64_t d3,
                               int64_t N1, int64_t N2, int64_t N3, float* dst)
{
    if (!src) {
        const IterState* st = c.st;
        if (st->done) return;
        const int cur = st->cur;
        src = sel == 0 ? c.x[cur] : sel == 1 ? c.x[cur ^ 1] : c.r[cur];
    }
    const int64_t n = N1 * N2 * N3;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k3 = i % N3, k2 = (i / N3) % N2, k1 = i / (N2 * N3);
        dst[i] = (k1 < d1 && k2 < d2 && k3 < d3) ? src[(k1 * d2 + k2) * d3 + k3] : 0.f;
    }
}

// spec *= hspec (forward) or conj(hspec) (adjoint); hspec already carries 1/prod(N).
__global__ void fft_mul_kernel(cufftComplex* spec, const cufftComplex* h, int64_t n, int adj, const IterState* st)
{
    if (st && st->done) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const cufftComplex a = spec[i], b = h[i];
        const float bi = adj ? -b.y : b.y;
        spec[i] = make_cuFloatComplex(a.x * b.x - a.y * bi, a.x * bi + a.y * b.x);
    }
}

// Plain operator output: the leading (d1, d2, d3) corner of the real grid.
__global__ void fft_crop_kernel(const float* src, int64_t d1, int64_t d2, int64_t d3, int64_t N2, int64_t N3,
                                float* out)
{
    const int64_t n = d1 * d2 * d3;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k3 = i % d3, k2 = (i / d3) % d2, k1 = i / (d2 * d3);
        out[i] = src[(k1 * N2 + k2) * N3 + k3];
    }
}

// Forward role: r = crop(A x) - y into r[cur] (initial) or r[cur ^ 1] (trial), partials of ||r||^2.
__global__ void __launch_bounds__(kEpiThreads) fft_residual_kernel(const float* src, IterCtx c, int init,
                                                                  int64_t b1, int64_t b2, int64_t b3, int64_t N2,
                                                                  int64_t N3)
{
    __shared__ double sh[kEpiThreads / 32];
    const IterState* st = c.st;
    if (st->done) return;
    const int cur = st->cur;
    float* r = init ? c.r[cur] : c.r[cur ^ 1];
    const int64_t n = b1 * b2 * b3;
    float loc = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k3 = i % b3, k2 = (i / b3) % b2, k1 = i / (b2 * b3);
        const float rr = src[(k1 * N2 + k2) * N3 + k3] - c.y[i];
        r[i] = rr;
        loc = fmaf(rr, rr, loc);
    }
    const double t = block_sum((double)loc, sh);
    if (threadIdx.x == 0) c.part_f[blockIdx.x] = t;
}

// Adjoint role: g = crop(A^T r) (fresh gradient only), x_t = max(x - delta (g + lambda x), 0) into
// x[cur ^ 1], partials of ||x_t - x||^2 and, when used, of the step-rule variants.
__global__ void __launch_bounds__(kEpiThreads) fft_update_kernel(const float* src, IterCtx c, int64_t m1,
                                                                int64_t m2, int64_t m3, int64_t N2, int64_t N3)
{
    __shared__ double sh[kEpiThreads / 32];
    const IterState* st = c.st;
    if (st->done) return;
    const int cur = st->cur;
    const bool fresh = st->need_grad != 0;
    const float delta = (float)st->delta, lamf = (float)st->lambda;
    const bool want_a = st->sigma != 0.0, want_x = st->lambda != 0.0;
    const bool want_sy = st->bb && fresh && st->accepted >= 1;
    const float* x = c.x[cur];
    float* xp = c.x[cur ^ 1];
    const int64_t n = m1 * m2 * m3;
    float loc = 0.f, loc_a = 0.f, loc_x = 0.f, loc_sy = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float xo = x[i];
        float gg;
        if (fresh) {
            const int64_t k3 = i % m3, k2 = (i / m3) % m2, k1 = i / (m2 * m3);
            gg = src[(k1 * N2 + k2) * N3 + k3];
            if (want_sy) {
                const float s = xo - xp[i];
                loc_sy = fmaf(s, fmaf(lamf, s, gg - c.g[i]), loc_sy);
            }
            c.g[i] = gg;
        } else {
            gg = c.g[i];
        }
        const float gt = fmaf(lamf, xo, gg);
        const float xn = fmaxf(fmaf(-delta, gt, xo), 0.f);
        xp[i] = xn;
        const float d = xn - xo;
        loc = fmaf(d, d, loc);
        loc_a = fmaf(gt, d, loc_a);
        loc_x = fmaf(xn, xn, loc_x);
    }
    double t = block_sum((double)loc, sh);
    if (threadIdx.x == 0) c.part_m[blockIdx.x] = t;
    if (want_a) {
        t = block_sum((double)loc_a, sh);
        if (threadIdx.x == 0) c.part_a[blockIdx.x] = t;
    }
    if (want_x) {
        t = block_sum((double)loc_x, sh);
        if (threadIdx.x == 0) c.part_x[blockIdx.x] = t;
    }
    if (want_sy) {
        t = block_sum((double)loc_sy, sh);
        if (threadIdx.x == 0) c.part_sy[blockIdx.x] = t;
    }
}

__global__ void fft_scale_kernel(cufftComplex* h, int64_t n, float a)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        h[i] = make_cuFloatComplex(h[i].x * a, h[i].y * a);
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

cudaError_t cufft_err(cufftResult r) { return r == CUFFT_SUCCESS ? cudaSuccess : cudaErrorUnknown; }

}  // namespace

int fft_epilogue_blocks() { return kEpiBlocks; }

cudaError_t fft_setup(FftPlan& F, const ConvGeom& gf, void* (*alloc)(void* owner, size_t bytes), void* owner)
{
    F.N[0] = good_size(gf.b1);
    F.N[1] = good_size(gf.b2);
    F.N[2] = good_size(gf.b3);
    F.nreal = F.N[0] * F.N[1] * F.N[2];
    F.ncplx = F.N[0] * F.N[1] * (F.N[2] / 2 + 1);
    if (F.N[0] > (1 << 30) || F.N[1] > (1 << 30) || F.N[2] > (1 << 30)) return cudaErrorInvalidValue;
    int dims[3] = {(int)F.N[0], (int)F.N[1], (int)F.N[2]};
    // leading axes of length 1 are dropped from the transform's rank
    int lead = 0;
    while (lead < 2 && dims[lead] == 1) lead++;
    const int rank = 3 - lead;
    if (cufftPlanMany(&F.r2c, rank, dims + lead, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, 1) != CUFFT_SUCCESS)
        return cudaErrorMemoryAllocation;
    if (cufftPlanMany(&F.c2r, rank, dims + lead, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, 1) != CUFFT_SUCCESS) {
        cufftDestroy(F.r2c);
        return cudaErrorMemoryAllocation;
    }
    F.have_plans = true;
    F.real = static_cast<float*>(alloc(owner, F.nreal * sizeof(float)));
    F.spec = alloc(owner, F.ncplx * sizeof(cufftComplex));
    F.hspec = alloc(owner, F.ncplx * sizeof(cufftComplex));
    if (!F.real || !F.spec || !F.hspec) return cudaErrorMemoryAllocation;
    return cudaSuccess;
}

void fft_release(FftPlan& F)
{
    if (F.have_plans) {
        cufftDestroy(F.r2c);
        cufftDestroy(F.c2r);
        F.have_plans = false;
    }
}

// Spectrum of the zero-padded template, scaled by 1/prod(N).
cudaError_t fft_set_psf(FftPlan& F, const float* H, int q1, int q2, int q3, cudaStream_t s)
{
    fft_pad_kernel<<<grid_for(F.nreal), 256, 0, s>>>(H, 0, IterCtx{}, q1, q2, q3, F.N[0], F.N[1], F.N[2], F.real);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = cufft_err(cufftSetStream(F.r2c, s))) != cudaSuccess) return e;
    if ((e = cufft_err(cufftExecR2C(F.r2c, F.real, static_cast<cufftComplex*>(F.hspec)))) != cudaSuccess) return e;
    // the 1/prod(N) of the unnormalised inverse transform, folded into the template's spectrum once
    fft_scale_kernel<<<grid_for(F.ncplx), 256, 0, s>>>(static_cast<cufftComplex*>(F.hspec), F.ncplx,
                                                       (float)(1.0 / (double)F.nreal));
    return cudaGetLastError();
}

// Plain operator: forward (m -> m + 2p) or adjoint (m + 2p -> m) of one volume.
cudaError_t fft_conv(FftPlan& F, const ConvGeom& g, bool fwd, const float* in, float* out, cudaStream_t s)
{
    fft_pad_kernel<<<grid_for(F.nreal), 256, 0, s>>>(in, 0, IterCtx{}, g.a1, g.a2, g.a3, F.N[0], F.N[1], F.N[2],
                                                     F.real);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cufftComplex* spec = static_cast<cufftComplex*>(F.spec);
    if ((e = cufft_err(cufftSetStream(F.r2c, s))) != cudaSuccess) return e;
    if ((e = cufft_err(cufftExecR2C(F.r2c, F.real, spec))) != cudaSuccess) return e;
    fft_mul_kernel<<<grid_for(F.ncplx), 256, 0, s>>>(spec, static_cast<const cufftComplex*>(F.hspec), F.ncplx,
                                                     fwd ? 0 : 1, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cufft_err(cufftSetStream(F.c2r, s))) != cudaSuccess) return e;
    if ((e = cufft_err(cufftExecC2R(F.c2r, spec, F.real))) != cudaSuccess) return e;
    fft_crop_kernel<<<grid_for(g.b1 * g.b2 * g.b3), 256, 0, s>>>(F.real, g.b1, g.b2, g.b3, F.N[1], F.N[2], out);
    return cudaGetLastError();
}

// Iteration roles.  fwd: input x[cur] (init) or x[cur ^ 1] (trial), residual into r[...]; adjoint:
// input r[cur], gradient and projected update.
cudaError_t fft_role(FftPlan& F, const ConvGeom& g, int role, const IterCtx& c, cudaStream_t s)
{
    const bool fwd = role == ROLE_FWD_INIT || role == ROLE_FWD_TRIAL;
    const int sel = role == ROLE_FWD_INIT ? 0 : role == ROLE_FWD_TRIAL ? 1 : 2;
    fft_pad_kernel<<<grid_for(F.nreal), 256, 0, s>>>(nullptr, sel, c, g.a1, g.a2, g.a3, F.N[0], F.N[1], F.N[2],
                                                     F.real);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cufftComplex* spec = static_cast<cufftComplex*>(F.spec);
    if ((e = cufft_err(cufftSetStream(F.r2c, s))) != cudaSuccess) return e;
    if ((e = cufft_err(cufftExecR2C(F.r2c, F.real, spec))) != cudaSuccess) return e;
    fft_mul_kernel<<<grid_for(F.ncplx), 256, 0, s>>>(spec, static_cast<const cufftComplex*>(F.hspec), F.ncplx,
                                                     fwd ? 0 : 1, c.st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cufft_err(cufftSetStream(F.c2r, s))) != cudaSuccess) return e;
    if ((e = cufft_err(cufftExecC2R(F.c2r, spec, F.real))) != cudaSuccess) return e;
    if (fwd)
        fft_residual_kernel<<<kEpiBlocks, kEpiThreads, 0, s>>>(F.real, c, role == ROLE_FWD_INIT ? 1 : 0, g.b1, g.b2,
                                                               g.b3, F.N[1], F.N[2]);
    else
        fft_update_kernel<<<kEpiBlocks, kEpiThreads, 0, s>>>(F.real, c, g.b1, g.b2, g.b3, F.N[1], F.N[2]);
    return cudaGetLastError();
}

}  // namespace cdv

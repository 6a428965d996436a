// The whole projected-gradient run of a small problem in one CTA.
//
// For volumes whose iterate, residuals, gradient and observation fit in one
// SM's shared memory (a 64x64 image with a 7x7 template needs ~120 KB), the
// K steps of Steps 1-3 run inside a single launch: no per-step kernel
// launches, no global-memory round trips, the step rule decided by thread 0
// between block barriers.  Semantics are those of the general path (same
// step rule, same FP64 objective and decisions, same report).
//
// Layout in shared memory (floats): the template; two iterates stored with a
// zero halo of 2p on every axis (so the forward's window loads need no bounds
// checks); the gradient; the observation and two residuals with a padded row
// pitch.  Lanes of a warp take consecutive rows.  Each thread computes 8 consecutive outputs along the contiguous axis
// with a register window (template width Q3 compile-time), and adds the taps
// of each template plane into a per-plane partial before the running total.
#include <math.h>

#include <algorithm>

#include "cdv_internal.h"

namespace cdv {

namespace {

constexpr int kSR = 8;          // outputs per thread job along the contiguous axis
constexpr int kSThreads = 512;

__host__ __device__ inline int c8(int v) { return (v + 7) & ~7; }

struct SmallLayout {
    int m1, m2, m3, p1, p2, p3, q1, q2, q3, n1, n2, n3;
    int xs1, xs2, xs3;          // padded iterate dims (m + 4p), row pitch xs3
    int rs3;                    // residual / observation row pitch
    int nh_pad, x_sz, r_sz, nx;
    size_t off_h, off_x0, off_x1, off_g, off_y, off_r0, off_r1, floats;
    __host__ __device__ static SmallLayout make(const int* m, const int* p)
    {
        SmallLayout L;
        L.m1 = m[0]; L.m2 = m[1]; L.m3 = m[2];
        L.p1 = p[0]; L.p2 = p[1]; L.p3 = p[2];
        L.q1 = 2 * p[0] + 1; L.q2 = 2 * p[1] + 1; L.q3 = 2 * p[2] + 1;
        L.n1 = L.m1 + 2 * L.p1; L.n2 = L.m2 + 2 * L.p2; L.n3 = L.m3 + 2 * L.p3;
        L.xs1 = L.m1 + 4 * L.p1;
        L.xs2 = L.m2 + 4 * L.p2;
        // Row pitches: long enough for the windows of the last job of a row, and odd, so
        // that the 32 lanes of a warp (32 consecutive rows) read 32 different banks.
        L.xs3 = (c8(L.n3) + L.q3 - 1) | 1;
        L.rs3 = (L.n3 > c8(L.m3) + L.q3 - 1 ? L.n3 : c8(L.m3) + L.q3 - 1) | 1;
        L.nh_pad = (L.q1 * L.q2 * L.q3 + 3) & ~3;
        L.x_sz = L.xs1 * L.xs2 * L.xs3;
        L.r_sz = L.n1 * L.n2 * L.rs3;
        L.nx = L.m1 * L.m2 * L.m3;
        L.off_h = 0;
        L.off_x0 = L.off_h + L.nh_pad;
        L.off_x1 = L.off_x0 + L.x_sz;
        L.off_g = L.off_x1 + L.x_sz;
        L.off_y = L.off_g + L.nx;
        L.off_r0 = L.off_y + L.r_sz;
        L.off_r1 = L.off_r0 + L.r_sz;
        L.floats = (L.off_r1 + L.r_sz + 1) & ~(size_t)1;
        return L;
    }
    __host__ __device__ size_t bytes() const { return floats * sizeof(float) + 64 * sizeof(double); }
};

struct SmallArgs {
    int m[3], p[3];
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

// Deterministic block sum: warp shuffles, then warp 0 adds the 32 warp sums in order.
__device__ double small_block_sum(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += red[i];
        red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// r = A x - y on the zero-haloed iterate xp; returns this thread's sum of r^2.
template <int Q3>
__device__ float small_forward(const SmallLayout& L, const float* __restrict__ h, const float* __restrict__ xp,
                                const float* __restrict__ y, float* __restrict__ r)
{
    constexpr int WL = kSR + Q3 - 1;
    const int blocks3 = (L.n3 + kSR - 1) / kSR;
    const int jobs = L.n1 * L.n2 * blocks3;
    float loc = 0.f;
    for (int job = threadIdx.x; job < jobs; job += blockDim.x) {
        const int s2 = job % L.n2, b3 = (job / L.n2) % blocks3, s1 = job / (blocks3 * L.n2);
        const int s3 = b3 * kSR;
        float tot[kSR];
#pragma unroll
        for (int c = 0; c < kSR; c++) tot[c] = 0.f;
        for (int j1 = 0; j1 < L.q1; j1++) {
            float part[kSR];
#pragma unroll
            for (int c = 0; c < kSR; c++) part[c] = 0.f;
            for (int j2 = 0; j2 < L.q2; j2++) {
                // padded row of x(s1 - j1, s2 - j2, .): index + 2p on every axis
                const float* row = xp + ((size_t)(s1 - j1 + 2 * L.p1) * L.xs2 + (s2 - j2 + 2 * L.p2)) * L.xs3 + s3;
                float w[WL];
#pragma unroll
                for (int t = 0; t < WL; t++) w[t] = row[t];
                const float* hr = h + (j1 * L.q2 + j2) * Q3;
#pragma unroll
                for (int j3 = 0; j3 < Q3; j3++) {
                    const float hv = hr[j3];
#pragma unroll
                    for (int c = 0; c < kSR; c++) part[c] = fmaf(hv, w[c + Q3 - 1 - j3], part[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < kSR; c++) tot[c] += part[c];
        }
#pragma unroll
        for (int c = 0; c < kSR; c++) {
            if (s3 + c < L.n3) {
                const size_t i = ((size_t)s1 * L.n2 + s2) * L.rs3 + s3 + c;
                const float rv = tot[c] - y[i];
                r[i] = rv;
                loc = fmaf(rv, rv, loc);
            }
        }
    }
    return loc;
}

// g = A^T r (valid correlation with the template).
template <int Q3>
__device__ void small_adjoint(const SmallLayout& L, const float* __restrict__ h, const float* __restrict__ r,
                              float* __restrict__ g)
{
    constexpr int WL = kSR + Q3 - 1;
    const int blocks3 = (L.m3 + kSR - 1) / kSR;
    const int jobs = L.m1 * L.m2 * blocks3;
    for (int job = threadIdx.x; job < jobs; job += blockDim.x) {
        const int k2 = job % L.m2, b3 = (job / L.m2) % blocks3, k1 = job / (blocks3 * L.m2);
        const int k3 = b3 * kSR;
        float tot[kSR];
#pragma unroll
        for (int c = 0; c < kSR; c++) tot[c] = 0.f;
        for (int j1 = 0; j1 < L.q1; j1++) {
            float part[kSR];
#pragma unroll
            for (int c = 0; c < kSR; c++) part[c] = 0.f;
            for (int j2 = 0; j2 < L.q2; j2++) {
                const float* row = r + ((size_t)(k1 + j1) * L.n2 + (k2 + j2)) * L.rs3 + k3;
                float w[WL];
#pragma unroll
                for (int t = 0; t < WL; t++) w[t] = row[t];
                const float* hr = h + (j1 * L.q2 + j2) * Q3;
#pragma unroll
                for (int j3 = 0; j3 < Q3; j3++) {
                    const float hv = hr[j3];
#pragma unroll
                    for (int c = 0; c < kSR; c++) part[c] = fmaf(hv, w[c + j3], part[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < kSR; c++) tot[c] += part[c];
        }
#pragma unroll
        for (int c = 0; c < kSR; c++)
            if (k3 + c < L.m3) g[((size_t)k1 * L.m2 + k2) * L.m3 + k3 + c] = tot[c];
    }
}

template <int Q3>
__global__ void __launch_bounds__(kSThreads, 1) small_iterate_kernel(const SmallArgs a)
{
    extern __shared__ __align__(16) float sm[];
    const SmallLayout L = SmallLayout::make(a.m, a.p);
    float* s_h = sm + L.off_h;
    float* s_x[2] = {sm + L.off_x0, sm + L.off_x1};
    float* s_g = sm + L.off_g;
    float* s_y = sm + L.off_y;
    float* s_r[2] = {sm + L.off_r0, sm + L.off_r1};
    double* red = reinterpret_cast<double*>(sm + L.floats);
    __shared__ int sh_ctl[4];          // cur, need_grad, done
    __shared__ double sh_delta;

    const int tid = threadIdx.x, nt = blockDim.x;
    for (size_t i = tid; i < L.floats; i += nt) sm[i] = 0.f;
    __syncthreads();
    const int nh = L.q1 * L.q2 * L.q3;
    for (int i = tid; i < nh; i += nt) s_h[i] = a.h[i];
    for (int i = tid; i < L.n1 * L.n2 * L.n3; i += nt) {
        const int c = i % L.n3, rr = i / L.n3;
        s_y[(size_t)rr * L.rs3 + c] = a.y[i];
    }
    __syncthreads();
    // x_0 into the interior of iterate 0 (Step 1)
    for (int i = tid; i < L.nx; i += nt) {
        const int k3 = i % L.m3, k2 = (i / L.m3) % L.m2, k1 = i / (L.m3 * L.m2);
        float v;
        if (a.x0_policy == CDV_X0_GIVEN) v = a.x[i];
        else if (a.x0_policy == CDV_X0_ZERO) v = 0.f;
        else {
            const float yy = s_y[((size_t)(k1 + L.p1) * L.n2 + (k2 + L.p2)) * L.rs3 + (k3 + L.p3)];
            v = yy > 0.f ? yy : 0.f;
        }
        s_x[0][((size_t)(k1 + 2 * L.p1) * L.xs2 + (k2 + 2 * L.p2)) * L.xs3 + (k3 + 2 * L.p3)] = v;
    }
    double delta0 = a.delta0;
    if (!(delta0 > 0.0)) {
        const double s = *a.absum;
        delta0 = 1.0 / (s * s);
    }
    __syncthreads();

    double F = 0.5 * small_block_sum((double)small_forward<Q3>(L, s_h, s_x[0], s_y, s_r[0]), red);
    // state kept by thread 0 in registers, published through shared memory
    double f_cur = F, delta = delta0;
    int accepted = 0, rejected = 0, halvings = 0, trials = 0, adj_convs = 0, status = CDV_OK;
    if (tid == 0) {
        a.f_hist[0] = F;
        sh_ctl[0] = 0;
        sh_ctl[1] = 1;
        sh_ctl[2] = (!isfinite(F) || a.K <= 0) ? 1 : 0;
        if (!isfinite(F)) status = CDV_ERR_NONFINITE;
        sh_delta = delta0;
    }
    __syncthreads();
    while (!sh_ctl[2]) {
        const int cur = sh_ctl[0];
        const int need_grad = sh_ctl[1];
        const double dl = sh_delta;
        if (need_grad) small_adjoint<Q3>(L, s_h, s_r[cur], s_g);
        __syncthreads();
        // projected update into the other iterate (Step 2); rows of the contiguous axis, no division
        float mv = 0.f;
        const float dlf = (float)dl;
        for (int row = tid / 32; row < L.m1 * L.m2; row += nt / 32) {
            const int k1 = row / L.m2, k2 = row - k1 * L.m2;
            const size_t xb = ((size_t)(k1 + 2 * L.p1) * L.xs2 + (k2 + 2 * L.p2)) * L.xs3 + 2 * L.p3;
            const float* gr = s_g + (size_t)row * L.m3;
            for (int k3 = tid & 31; k3 < L.m3; k3 += 32) {
                const float xo = s_x[cur][xb + k3];
                const float xn = fmaxf(fmaf(-dlf, gr[k3], xo), 0.f);
                s_x[cur ^ 1][xb + k3] = xn;
                const float d = xn - xo;
                mv = fmaf(d, d, mv);
            }
        }
        __syncthreads();
        const double M = small_block_sum((double)mv, red);
        const double Ft =
            0.5 * small_block_sum((double)small_forward<Q3>(L, s_h, s_x[cur ^ 1], s_y, s_r[cur ^ 1]), red);
        if (tid == 0) {
            trials++;
            if (need_grad) adj_convs++;
            int done = 0;
            if (M == 0.0) {
                status = CDV_ERR_NOT_DESCENDING;
                done = 1;
            } else if (!isfinite(Ft)) {
                status = CDV_ERR_NONFINITE;
                done = 1;
            } else if (Ft < f_cur) {
                if (accepted < a.hist_cap) {
                    a.d_hist[accepted] = dl;
                    a.f_hist[accepted + 1] = Ft;
                }
                accepted++;
                f_cur = Ft;
                halvings = 0;
                delta = delta0;
                sh_ctl[0] = cur ^ 1;
                sh_ctl[1] = 1;
                if (accepted >= a.K) done = 1;
            } else {
                rejected++;
                halvings++;
                sh_ctl[1] = 0;
                if (halvings > a.max_halvings || rejected > a.max_rejects) {
                    status = CDV_ERR_NOT_DESCENDING;
                    done = 1;
                } else {
                    delta *= a.beta;
                }
            }
            sh_delta = delta;
            sh_ctl[2] = done;
        }
        __syncthreads();
    }
    const int cur = sh_ctl[0];
    for (int i = tid; i < L.nx; i += nt) {
        const int k3 = i % L.m3, k2 = (i / L.m3) % L.m2, k1 = i / (L.m3 * L.m2);
        a.x[i] = s_x[cur][((size_t)(k1 + 2 * L.p1) * L.xs2 + (k2 + 2 * L.p2)) * L.xs3 + (k3 + 2 * L.p3)];
    }
    if (tid == 0) {
        IterState* st = a.st;
        st->f_cur = f_cur;
        st->f_trial = f_cur;
        st->delta = delta;
        st->delta0 = delta0;
        st->beta = a.beta;
        st->moved = 0.0;
        st->accepted = accepted;
        st->rejected = rejected;
        st->halvings = halvings;
        st->max_halvings = a.max_halvings;
        st->max_rejects = a.max_rejects;
        st->K = a.K;
        st->cur = 0;
        st->need_grad = 0;
        st->done = 1;
        st->status = status;
        st->trials = trials;
        st->hist_cap = a.hist_cap;
        st->adj_convs = adj_convs;
    }
}

template <int Q3>
cudaError_t small_prepare()
{
    return cudaFuncSetAttribute(small_iterate_kernel<Q3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
}

}  // namespace

size_t small_smem_bytes(const int64_t* m, const int* p)
{
    int mi[3] = {(int)m[0], (int)m[1], (int)m[2]};
    return SmallLayout::make(mi, p).bytes();
}

bool small_supported(const int64_t* m, const int* p)
{
    const int q3 = 2 * p[2] + 1;
    if (q3 > 15) return false;
    if (m[0] > 4096 || m[1] > 4096 || m[2] > 4096) return false;
    return small_smem_bytes(m, p) <= 200 * 1024;
}

cudaError_t small_iterate(const SmallRun& r, cudaStream_t s, bool prepare)
{
    SmallArgs a;
    for (int i = 0; i < 3; i++) {
        a.m[i] = (int)r.m[i];
        a.p[i] = r.p[i];
    }
    a.y = r.y;
    a.x = r.x;
    a.h = r.h;
    a.st = r.st;
    a.f_hist = r.f_hist;
    a.d_hist = r.d_hist;
    a.hist_cap = r.hist_cap;
    a.K = r.K;
    a.x0_policy = r.x0_policy;
    a.max_halvings = r.max_halvings;
    a.max_rejects = r.max_rejects;
    a.delta0 = r.delta0;
    a.beta = r.beta;
    a.absum = r.absum;
    const size_t smem = small_smem_bytes(r.m, r.p);
    const int q3 = 2 * r.p[2] + 1;
    if (prepare) {
        switch (q3) {
        case 1: return small_prepare<1>();
        case 3: return small_prepare<3>();
        case 5: return small_prepare<5>();
        case 7: return small_prepare<7>();
        case 9: return small_prepare<9>();
        case 11: return small_prepare<11>();
        case 13: return small_prepare<13>();
        case 15: return small_prepare<15>();
        default: return cudaErrorInvalidValue;
        }
    }
    void* args[] = {&a};
    const void* fn = nullptr;
    switch (q3) {
    case 1: fn = (const void*)small_iterate_kernel<1>; break;
    case 3: fn = (const void*)small_iterate_kernel<3>; break;
    case 5: fn = (const void*)small_iterate_kernel<5>; break;
    case 7: fn = (const void*)small_iterate_kernel<7>; break;
    case 9: fn = (const void*)small_iterate_kernel<9>; break;
    case 11: fn = (const void*)small_iterate_kernel<11>; break;
    case 13: fn = (const void*)small_iterate_kernel<13>; break;
    case 15: fn = (const void*)small_iterate_kernel<15>; break;
    default: return cudaErrorInvalidValue;
    }
    return cudaLaunchKernel(fn, dim3(1), dim3(kSThreads), args, smem, s);
}

}  // namespace cdv

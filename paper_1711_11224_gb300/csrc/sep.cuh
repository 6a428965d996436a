// Separable-template engine (CDV_MODE_SEPARABLE): the two operators of a template that is an outer
// product H(j1, j2, j3) = h1(j1) h2(j2) h3(j3).
//
// The sum of Property 1 then factorises axis by axis: the n-D block-Toeplitz matrix A_n^h is the
// Kronecker product of the 1-D Toeplitz matrices of h1, h2, h3 (Property 1 applied to a template
// whose every block is a multiple of one (n-1)-D template), so
//   forward  Y = X (*) H       = three 1-D full convolutions (m_i -> m_i + 2p_i), axis 3, 2, then 1;
//   adjoint  G = M_2p(R (*) H~) = three 1-D valid correlations (m_i + 2p_i -> m_i), axis 1, 2, then 3,
// each pass computing, over a volume viewed as (outer, kin, inner),
//   out[u, s, i] = sum_{j < Q} w[j] in[u, s + o - j, i]      (in = 0 outside [0, kin))
// with w = h_k, o = 0 (forward) or w = flipped h_k, o = 2p_k (adjoint).  The MACs per output drop
// from q1 q2 q3 to q1 + q2 + q3, and each pass is a stream over memory: the engine is bound by HBM
// (or L2) bandwidth, not by arithmetic.
//
// Two kernels:
//  * rows (the contiguous axis): a block stages rb rows x (seg + Q - 1) input samples in shared
//    memory with coalesced loads, each thread slides a register window over 7 outputs (7 is odd:
//    threads at a stride of 7 floats read distinct banks), the outputs go through shared memory and
//    leave coalesced;
//  * cols (a strided axis): lanes along the contiguous inner index (coalesced), each warp walks a
//    strip of outputs along the pass axis with a register window, so every input sample of the strip
//    is loaded once.
// The last pass of a direction carries the iteration's epilogue (residual, or projected update with
// the step-rule partial sums), so the fused roles match the direct engines'.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cdv_internal.h"

namespace cdv {

constexpr int kSepThreads = 256;
constexpr int kSepRowC = 7;       // outputs per thread of the rows kernel
constexpr int kSepColC = 8;       // outputs per window step of the cols kernel
constexpr int kSepBatch = 8;      // elements per thread whose loads are issued before any store

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f)
{
    const uint32_t t = __umulhi(f.m, n);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

__device__ __forceinline__ double sep_block_sum(double v, double* sh)
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

// Output side of one pass: a plain store (intermediate passes, plain operators) or the iteration
// epilogue of the direction's last pass.
struct SepEpi {
    int role;
    bool fresh, want_a, want_x, want_sy;
    float delta, lam;
    float* out;          // plain: output; forward roles: residual buffer
    const float* y;
    const float* x;      // adjoint role: x_k
    float* xp;           // adjoint role: x_trial (holds x_{k-1} on entry)
    float* g;
    float f, m, a, xx, sy;

    // N outputs (ok[i] false: skipped): every load of the batch is issued before its first store, so a
    // thread keeps N requests in flight instead of waiting on each in turn.  Used by the rows kernel,
    // which ends every adjoint (the cols kernel writes its forward residual itself).
    template <int N>
    __device__ __forceinline__ void put_batch(const int64_t (&idx)[N], const float (&v)[N], const bool (&ok)[N])
    {
        if (role == ROLE_PLAIN) {
#pragma unroll
            for (int i = 0; i < N; i++)
                if (ok[i]) out[idx[i]] = v[i];
            return;
        }
        if (role != ROLE_ADJ_TRIAL) {
            float yv[N];
#pragma unroll
            for (int i = 0; i < N; i++) yv[i] = ok[i] ? y[idx[i]] : 0.f;
#pragma unroll
            for (int i = 0; i < N; i++)
                if (ok[i]) {
                    const float rr = v[i] - yv[i];
                    out[idx[i]] = rr;
                    f = fmaf(rr, rr, f);
                }
            return;
        }
        const bool need_old = !fresh || want_sy;
        float xo[N], xq[N], go[N];
#pragma unroll
        for (int i = 0; i < N; i++) {
            xo[i] = ok[i] ? x[idx[i]] : 0.f;
            xq[i] = (ok[i] && want_sy) ? xp[idx[i]] : 0.f;
            go[i] = (ok[i] && need_old) ? g[idx[i]] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < N; i++) {
            if (!ok[i]) continue;
            float gg = v[i];
            if (fresh) {
                if (want_sy) {                               // before g and x_{k-1} are overwritten
                    const float sd = xo[i] - xq[i];
                    sy = fmaf(sd, fmaf(lam, sd, gg - go[i]), sy);
                }
                g[idx[i]] = gg;
            } else {
                gg = go[i];
            }
            const float gt = fmaf(lam, xo[i], gg);          // grad f = A^T r + lambda x
            const float xn = fmaxf(fmaf(-delta, gt, xo[i]), 0.f);
            xp[idx[i]] = xn;
            const float d = xn - xo[i];
            m = fmaf(d, d, m);
            a = fmaf(gt, d, a);
            xx = fmaf(xn, xn, xx);
        }
    }

    // FP64 block partials of the sums (one entry per block of the launch).
    __device__ __forceinline__ void finish(const IterCtx& c, double* sh)
    {
        if (role == ROLE_PLAIN) return;
        if (role != ROLE_ADJ_TRIAL) {
            const double t = sep_block_sum((double)f, sh);
            if (threadIdx.x == 0) c.part_f[blockIdx.x] = t;
            return;
        }
        double t = sep_block_sum((double)m, sh);
        if (threadIdx.x == 0) c.part_m[blockIdx.x] = t;
        if (want_a) {
            t = sep_block_sum((double)a, sh);
            if (threadIdx.x == 0) c.part_a[blockIdx.x] = t;
        }
        if (want_x) {
            t = sep_block_sum((double)xx, sh);
            if (threadIdx.x == 0) c.part_x[blockIdx.x] = t;
        }
        if (want_sy) {
            t = sep_block_sum((double)sy, sh);
            if (threadIdx.x == 0) c.part_sy[blockIdx.x] = t;
        }
    }
};

// Input, output and epilogue of one pass under its role.  Returns false when the launch has nothing
// to do (the run has finished, or an adjoint pass whose gradient is reused); `conv` is false for the
// last adjoint pass of a trial that reuses the gradient (update only).
__device__ __forceinline__ bool sep_begin(const SepPass& P, const float*& in, SepEpi& e, bool& conv)
{
    in = P.in;
    conv = true;
    e = SepEpi{};
    e.role = P.last ? P.role : (int)ROLE_PLAIN;
    e.out = P.out;
    if (P.role == ROLE_PLAIN) return true;
    const IterState* st = P.c.st;
    if (st->done) return false;                          // uniform: the run has finished
    const int cur = st->cur;
    if (P.role == ROLE_FWD_INIT || P.role == ROLE_FWD_TRIAL) {
        const int b = P.role == ROLE_FWD_INIT ? cur : cur ^ 1;
        if (P.first) in = P.c.x[b];
        if (P.last) e.out = P.c.r[b];
        e.y = P.c.y;
        return true;
    }
    conv = st->need_grad != 0;
    if (!conv && !P.last) return false;
    if (P.first) in = P.c.r[cur];
    e.fresh = conv;
    e.delta = (float)st->delta;
    e.lam = (float)st->lambda;
    e.want_a = st->sigma != 0.0;
    e.want_x = st->lambda != 0.0;
    e.want_sy = st->bb && conv && st->accepted >= 1;
    e.x = P.c.x[cur];
    e.xp = P.c.x[cur ^ 1];
    e.g = P.c.g;
    return true;
}

// Update-only form of the last adjoint pass (the trial reuses g).
__device__ __forceinline__ void sep_update_only(const SepPass& P, SepEpi& e)
{
    const int64_t n = P.outer * P.kout * P.inner;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += stride * kSepBatch) {
        int64_t idx[kSepBatch];
        float v[kSepBatch];
        bool ok[kSepBatch];
#pragma unroll
        for (int u = 0; u < kSepBatch; u++) {
            idx[u] = i0 + u * stride;
            ok[u] = idx[u] < n;
            v[u] = 0.f;
        }
        e.put_batch<kSepBatch>(idx, v, ok);
    }
}

// Pass along the contiguous axis (inner == 1): `outer` rows of kin samples -> rows of kout samples.
// EPI false: plain stores only (intermediate passes and plain operators: fewer registers, more blocks
// per SM); true: every role of a direction's last pass.
template <int Q, bool EPI>
__global__ void __launch_bounds__(kSepThreads) sep_rows_kernel(const SepPass P)
{
    constexpr int C = kSepRowC;
    constexpr int WN = C + Q - 1;
    extern __shared__ float sm[];
    __shared__ double sh[kSepThreads / 32];
    const float* in;
    SepEpi e;
    bool conv;
    if (!sep_begin(P, in, e, conv)) return;
    if (EPI && !conv) {
        sep_update_only(P, e);
        e.finish(P.c, sh);
        return;
    }
    float w[Q];
#pragma unroll
    for (int j = 0; j < Q; j++) w[j] = P.w[j];
    const int tid = threadIdx.x;
    const int seg = P.seg, rb = P.rb;
    const int span = seg + Q - 1;
    const int pitch = span | 1;                          // odd: consecutive rows start on other banks
    float* s_in = sm;                                    // rb x pitch
    float* s_out = sm + rb * pitch;                      // rb x seg
    const int cpr = seg / C;
    const int64_t nrows = P.outer;
    const int64_t nseg = (P.kout + seg - 1) / seg;
    const int64_t ntask = ((nrows + rb - 1) / rb) * nseg;
    // row strides for tasks of several rows (rows shorter than 256 * 7 samples); a task of one row
    // (r = 0) may be longer than 2^31 samples
    const int kin = rb > 1 ? (int)P.kin : 0, kout = rb > 1 ? (int)P.kout : 0;
    for (int64_t task = blockIdx.x; task < ntask; task += gridDim.x) {
        const int64_t row0 = (task / nseg) * rb;
        const int64_t s0 = (task % nseg) * seg;
        const int64_t t0 = s0 + P.o - (Q - 1);           // input sample of shared column 0
        // 32-bit offsets from per-task bases (r * kin and r * kout stay far below 2^31)
        const int rows = (int)(nrows - row0 < rb ? nrows - row0 : rb);
        const int xlo = (int)(t0 < 0 ? -t0 : 0);                      // columns whose sample is in [0, kin)
        const int xhi = (int)(P.kin - t0 < span ? P.kin - t0 : span);
        const float* tin = in + row0 * P.kin + t0;
        for (int i0 = tid; i0 < rb * span; i0 += kSepThreads * kSepBatch) {
            float v[kSepBatch];
            int so[kSepBatch];
#pragma unroll
            for (int u = 0; u < kSepBatch; u++) {
                const int i = i0 + u * kSepThreads;
                const int r = (int)fdiv((uint32_t)i, P.dspan), xcol = i - r * span;
                so[u] = i < rb * span ? r * pitch + xcol : -1;
                v[u] = (so[u] >= 0 && r < rows && xcol >= xlo && xcol < xhi) ? tin[r * kin + xcol] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kSepBatch; u++)
                if (so[u] >= 0) s_in[so[u]] = v[u];
        }
        __syncthreads();
        for (int it = tid; it < rb * cpr; it += kSepThreads) {
            const int r = (int)fdiv((uint32_t)it, P.dcpr), cc = it - r * cpr;
            const float* src = s_in + r * pitch + cc * C;
            float v[WN];
#pragma unroll
            for (int k = 0; k < WN; k++) v[k] = src[k];
            float acc[C];
#pragma unroll
            for (int c = 0; c < C; c++) acc[c] = 0.f;
#pragma unroll
            for (int j = 0; j < Q; j++)                      // C independent chains, interleaved
#pragma unroll
                for (int c = 0; c < C; c++) acc[c] = fmaf(w[j], v[c + Q - 1 - j], acc[c]);
#pragma unroll
            for (int c = 0; c < C; c++) s_out[r * seg + cc * C + c] = acc[c];
        }
        __syncthreads();
        // coalesced along the row; the next task's staging touches s_in only, and its compute loop
        // writes s_out after the barrier that follows that staging
        const int xout = (int)(P.kout - s0 < seg ? P.kout - s0 : seg);    // outputs of the segment in the row
        const int64_t obase = row0 * P.kout + s0;
        for (int i0 = tid; i0 < rb * seg; i0 += kSepThreads * kSepBatch) {
            int off[kSepBatch];
            float v[kSepBatch];
            bool ok[kSepBatch];
#pragma unroll
            for (int u = 0; u < kSepBatch; u++) {
                const int i = i0 + u * kSepThreads;
                const int r = (int)fdiv((uint32_t)i, P.dseg), xcol = i - r * seg;
                ok[u] = i < rb * seg && r < rows && xcol < xout;
                off[u] = r * kout + xcol;
                v[u] = ok[u] ? s_out[i] : 0.f;
            }
            if (EPI) {
                int64_t idx[kSepBatch];
#pragma unroll
                for (int u = 0; u < kSepBatch; u++) idx[u] = obase + off[u];
                e.put_batch<kSepBatch>(idx, v, ok);
            } else {
                float* o = e.out + obase;
#pragma unroll
                for (int u = 0; u < kSepBatch; u++)
                    if (ok[u]) o[off[u]] = v[u];
            }
        }
    }
    if (EPI) e.finish(P.c, sh);
}

// Pass along a strided axis: (outer, kin, inner) -> (outer, kout, inner).  A warp task is 32
// consecutive inner positions x a strip of outputs along the pass axis.  EPI: the forward residual
// (the only role that ends in this kernel: the adjoint's last pass runs along the contiguous axis).
template <int Q, bool EPI>
__global__ void __launch_bounds__(kSepThreads) sep_cols_kernel(const SepPass P)
{
    constexpr int C = kSepColC;
    constexpr int WN = C + Q - 1;
    __shared__ double sh[kSepThreads / 32];
    const float* in;
    SepEpi e;
    bool conv;
    if (!sep_begin(P, in, e, conv) || !conv) return;     // !conv: a reused gradient (rows kernel's update)
    float w[Q];
#pragma unroll
    for (int j = 0; j < Q; j++) w[j] = P.w[j];
    const int lane = threadIdx.x & 31;
    constexpr int kWarps = kSepThreads / 32;
    const int64_t inner = P.inner, kin = P.kin, kout = P.kout;
    const int64_t nic = (inner + 31) / 32;
    const int64_t nstrip = (kout + P.strip - 1) / P.strip;
    const int64_t ntask = P.outer * nic * nstrip;
    for (int64_t t = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); t < ntask; t += (int64_t)gridDim.x * kWarps) {
        const int64_t ic = t % nic;                      // inner chunk fastest: neighbouring warps, neighbouring memory
        const int64_t rest = t / nic;
        const int64_t sp = rest % nstrip;
        const int64_t ou = rest / nstrip;
        const int64_t ii = ic * 32 + lane;
        const bool on = ii < inner;
        const int64_t sb = sp * P.strip;
        const int64_t se = sb + P.strip < kout ? sb + P.strip : kout;
        const float* base = in + ou * kin * inner + (on ? ii : 0);
        float v[WN];
        const int64_t tb = sb + P.o - (Q - 1);
#pragma unroll
        for (int k = 0; k < Q - 1; k++) {
            const int64_t tt = tb + k;
            v[k] = (on && tt >= 0 && tt < kin) ? base[tt * inner] : 0.f;
        }
        // the C input samples of a step are loaded one step ahead (into nx), so that their latency
        // overlaps the previous step's FMAs; the pointer walks the pass axis and is dereferenced only
        // inside [0, kin) (off lanes read column 0)
        float nx[C];
        auto load_step = [&](int64_t s) {
            const int64_t ts = s + P.o;
            const float* lp = base + ts * inner;
            if (ts >= 0 && ts + C <= kin) {
#pragma unroll
                for (int c = 0; c < C; c++) {
                    nx[c] = *lp;
                    lp += inner;
                }
            } else {
#pragma unroll
                for (int c = 0; c < C; c++) {
                    const int64_t tt = ts + c;
                    nx[c] = (on && tt >= 0 && tt < kin) ? *lp : 0.f;
                    lp += inner;
                }
            }
        };
        if (sb < se) load_step(sb);
        for (int64_t s = sb; s < se; s += C) {
#pragma unroll
            for (int c = 0; c < C; c++) v[Q - 1 + c] = nx[c];
            if (s + C < se) load_step(s + C);
            float acc[C];
#pragma unroll
            for (int c = 0; c < C; c++) acc[c] = 0.f;
#pragma unroll
            for (int j = 0; j < Q; j++)                      // C independent chains, interleaved
#pragma unroll
                for (int c = 0; c < C; c++) acc[c] = fmaf(w[j], v[c + Q - 1 - j], acc[c]);
            const int64_t off = (ou * kout + s) * inner + ii;
            if (EPI) {                                       // forward residual: r = A x - y
                float yv[C];
                const float* yp = e.y + off;
#pragma unroll
                for (int c = 0; c < C; c++) {                // independent of the FMAs: free to be issued early
                    yv[c] = (on && s + c < se) ? *yp : 0.f;
                    yp += inner;
                }
                float* rp = e.out + off;
#pragma unroll
                for (int c = 0; c < C; c++) {
                    if (on && s + c < se) {
                        const float rr = acc[c] - yv[c];
                        *rp = rr;
                        e.f = fmaf(rr, rr, e.f);
                    }
                    rp += inner;
                }
            } else {
                float* op = e.out + off;
#pragma unroll
                for (int c = 0; c < C; c++) {
                    if (on && s + c < se) *op = acc[c];
                    op += inner;
                }
            }
#pragma unroll
            for (int k = 0; k < Q - 1; k++) v[k] = v[k + C];
        }
    }
    if (EPI) e.finish(P.c, sh);
}

// EPI: the pass ends a role launch (its epilogue is more than a plain store).
template <int Q, bool EPI>
cudaError_t sep_launch_q(const SepPass& P, int blocks, cudaStream_t s)
{
    if (P.inner == 1) {
        const int span = P.seg + Q - 1;
        const size_t smem = (size_t)P.rb * ((span | 1) + P.seg) * sizeof(float);
        sep_rows_kernel<Q, EPI><<<blocks, kSepThreads, smem, s>>>(P);
    } else {
        sep_cols_kernel<Q, EPI><<<blocks, kSepThreads, 0, s>>>(P);
    }
    return cudaGetLastError();
}

}  // namespace cdv

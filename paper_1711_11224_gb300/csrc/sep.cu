// Host side of the separable-template engine: pass geometry, factor upload and launches.
//
// Forward (X: m -> Y: m + 2p), passes along axis 3, 2, 1:
//   X (m1 m2 rows x m3)        -> tA (m1, m2, m3 + 2p3)
//   tA (m1, m2 | m3 + 2p3)     -> tB (m1, m2 + 2p2, m3 + 2p3)
//   tB (m1 | (m2 + 2p2)(..))   -> Y                               (epilogue: residual)
// Adjoint (R: m + 2p -> G: m), passes along axis 1, 2, 3:
//   R                          -> tA (m1, m2 + 2p2, m3 + 2p3)
//   tA                         -> tB (m1, m2, m3 + 2p3)
//   tB (m1 m2 rows x m3 + 2p3) -> G                               (epilogue: projected update)
#include <algorithm>

#include "sep.cuh"

namespace cdv {

#define CDV_SEP_EXTERN(Q)                                                            \
    extern template cudaError_t sep_launch_q<Q, false>(const SepPass&, int, cudaStream_t); \
    extern template cudaError_t sep_launch_q<Q, true>(const SepPass&, int, cudaStream_t);
CDV_SEP_EXTERN(1) CDV_SEP_EXTERN(3) CDV_SEP_EXTERN(5) CDV_SEP_EXTERN(7) CDV_SEP_EXTERN(9) CDV_SEP_EXTERN(11)
CDV_SEP_EXTERN(13) CDV_SEP_EXTERN(15) CDV_SEP_EXTERN(17) CDV_SEP_EXTERN(19) CDV_SEP_EXTERN(21) CDV_SEP_EXTERN(23)
CDV_SEP_EXTERN(25) CDV_SEP_EXTERN(27) CDV_SEP_EXTERN(29) CDV_SEP_EXTERN(31)
#undef CDV_SEP_EXTERN

namespace {

constexpr int kSepBlocks = 152 * 8;

__global__ void sep_outer_kernel(const float* hf, int q1, int q2, int q3, float* H)
{
    const int n = q1 * q2 * q3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j3 = i % q3, j2 = (i / q3) % q2, j1 = i / (q2 * q3);
        H[i] = hf[j1] * hf[q1 + j2] * hf[q1 + q2 + j3];
    }
}

__global__ void sep_flip_kernel(const float* hf, float* hb, int q1, int q2, int q3)
{
    const int n = q1 + q2 + q3;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int a = i < q1 ? 0 : i < q1 + q2 ? 1 : 2;
        const int off = a == 0 ? 0 : a == 1 ? q1 : q1 + q2;
        const int q = a == 0 ? q1 : a == 1 ? q2 : q3;
        hb[i] = hf[off + q - 1 - (i - off)];
    }
}

__global__ void sep_one_kernel(float* h) { *h = 1.f; }

cudaError_t launch_pass(const SepPass& P, cudaStream_t s)
{
    const bool epi = P.last && P.role != ROLE_PLAIN;
    switch (P.q) {
#define CDV_CASE(Q) \
    case Q: return epi ? sep_launch_q<Q, true>(P, kSepBlocks, s) : sep_launch_q<Q, false>(P, kSepBlocks, s);
        CDV_CASE(1) CDV_CASE(3) CDV_CASE(5) CDV_CASE(7) CDV_CASE(9) CDV_CASE(11) CDV_CASE(13) CDV_CASE(15)
        CDV_CASE(17) CDV_CASE(19) CDV_CASE(21) CDV_CASE(23) CDV_CASE(25) CDV_CASE(27) CDV_CASE(29) CDV_CASE(31)
#undef CDV_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

// Work shape of a pass: rows kernel (inner == 1) -- one window of 7 outputs per thread, rows packed
// into a block task when they are short; cols kernel -- strips short enough to give about 48 warp
// tasks per SM, at least one window step long.
void shape(SepPass& P)
{
    if (P.inner == 1) {
        const int64_t full = (int64_t)kSepThreads * kSepRowC;
        const int64_t kr = (P.kout + kSepRowC - 1) / kSepRowC * kSepRowC;
        P.seg = (int)std::min<int64_t>(kr, full);
        P.rb = (int)std::max<int64_t>(1, std::min<int64_t>(full / P.seg, P.outer));
        P.strip = 0;
        P.dspan = make_fastdiv((uint32_t)(P.seg + P.q - 1));
        P.dcpr = make_fastdiv((uint32_t)(P.seg / kSepRowC));
        P.dseg = make_fastdiv((uint32_t)P.seg);
    } else {
        const int64_t lines = P.outer * ((P.inner + 31) / 32);
        const int64_t want = 152 * 48;
        const int64_t steps = (P.kout + kSepColC - 1) / kSepColC;
        const int64_t nstrip = std::max<int64_t>(1, std::min<int64_t>(steps, (want + lines - 1) / lines));
        P.strip = (steps + nstrip - 1) / nstrip * kSepColC;
        P.seg = P.rb = 0;
    }
}

SepPass make_pass(const float* w, int q, int o, int64_t outer, int64_t kin, int64_t kout, int64_t inner)
{
    SepPass P{};
    P.w = w;
    P.q = q;
    P.o = o;
    P.outer = outer;
    P.kin = kin;
    P.kout = kout;
    P.inner = inner;
    shape(P);
    return P;
}

}  // namespace

FastDiv make_fastdiv(uint32_t d)
{
    // l = ceil(log2 d); m = floor(2^32 (2^l - d) / d) + 1 (below 2^32 for every d >= 1)
    int l = 0;
    while (l < 32 && (1ull << l) < d) l++;
    FastDiv f;
    f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}

int sep_blocks() { return kSepBlocks; }

bool sep_supported(const int q[3])
{
    for (int a = 0; a < 3; a++)
        if (q[a] < 1 || q[a] > 31 || !(q[a] & 1)) return false;
    return true;
}

cudaError_t sep_setup(SepPlan& S, const int64_t m[3], const int p[3], void* (*alloc)(void* owner, size_t bytes),
                      void* owner)
{
    int q[3];
    int64_t b[3];
    for (int a = 0; a < 3; a++) {
        q[a] = 2 * p[a] + 1;
        b[a] = m[a] + 2 * p[a];
    }
    if (!sep_supported(q)) return cudaErrorInvalidValue;
    const int nq = q[0] + q[1] + q[2];
    S.hf = static_cast<float*>(alloc(owner, nq * sizeof(float)));
    S.hb = static_cast<float*>(alloc(owner, nq * sizeof(float)));
    const size_t nt = (size_t)m[0] * b[1] * b[2];
    S.tA = static_cast<float*>(alloc(owner, nt * sizeof(float)));
    S.tB = static_cast<float*>(alloc(owner, nt * sizeof(float)));
    if (!S.hf || !S.hb || !S.tA || !S.tB) return cudaErrorMemoryAllocation;
    const float* hf[3] = {S.hf, S.hf + q[0], S.hf + q[0] + q[1]};
    const float* hb[3] = {S.hb, S.hb + q[0], S.hb + q[0] + q[1]};
    S.fwd[0] = make_pass(hf[2], q[2], 0, m[0] * m[1], m[2], b[2], 1);
    S.fwd[1] = make_pass(hf[1], q[1], 0, m[0], m[1], b[1], b[2]);
    S.fwd[2] = make_pass(hf[0], q[0], 0, 1, m[0], b[0], b[1] * b[2]);
    S.adj[0] = make_pass(hb[0], q[0], 2 * p[0], 1, b[0], m[0], b[1] * b[2]);
    S.adj[1] = make_pass(hb[1], q[1], 2 * p[1], m[0], b[1], m[1], b[2]);
    S.adj[2] = make_pass(hb[2], q[2], 2 * p[2], m[0] * m[1], b[2], m[2], 1);
    for (SepPass* d : {S.fwd, S.adj}) {
        d[0].in = nullptr;
        d[0].out = S.tA;
        d[1].in = S.tA;
        d[1].out = S.tB;
        d[2].in = S.tB;
        d[2].out = nullptr;
        d[0].first = 1;
        d[2].last = 1;
    }
    // the projected-update epilogue exists in the rows kernel only
    if (S.adj[2].inner != 1) return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t sep_set_factors(SepPlan& S, const float* const h[3], const int q[3], float* H, cudaStream_t s)
{
    int off = 0;
    for (int a = 0; a < 3; a++) {
        cudaError_t e;
        if (h[a])
            e = cudaMemcpyAsync(S.hf + off, h[a], q[a] * sizeof(float), cudaMemcpyDeviceToDevice, s);
        else {
            sep_one_kernel<<<1, 1, 0, s>>>(S.hf + off);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return e;
        off += q[a];
    }
    sep_flip_kernel<<<1, 128, 0, s>>>(S.hf, S.hb, q[0], q[1], q[2]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n = q[0] * q[1] * q[2];
    sep_outer_kernel<<<std::min((n + 255) / 256, 1024), 256, 0, s>>>(S.hf, q[0], q[1], q[2], H);
    return cudaGetLastError();
}

cudaError_t sep_conv(const SepPlan& S, bool fwd, const float* in, float* out, cudaStream_t s)
{
    const SepPass* d = fwd ? S.fwd : S.adj;
    for (int i = 0; i < 3; i++) {
        SepPass P = d[i];
        P.role = ROLE_PLAIN;
        if (i == 0) P.in = in;
        if (i == 2) P.out = out;
        const cudaError_t e = launch_pass(P, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t sep_role(const SepPlan& S, bool fwd, int role, const IterCtx& c, cudaStream_t s)
{
    const SepPass* d = fwd ? S.fwd : S.adj;
    for (int i = 0; i < 3; i++) {
        SepPass P = d[i];
        P.role = role;
        P.c = c;
        const cudaError_t e = launch_pass(P, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

double sep_pass_macs(const SepPlan& S, bool fwd)
{
    const SepPass* d = fwd ? S.fwd : S.adj;
    double t = 0.0;
    for (int i = 0; i < 3; i++) t += (double)d[i].outer * (double)d[i].kout * (double)d[i].inner * d[i].q;
    return t;
}

}  // namespace cdv

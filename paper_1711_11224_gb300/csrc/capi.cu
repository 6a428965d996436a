// C ABI of libcdv: plans, the forward/adjoint operators, the template
// gradient, the projected-gradient iteration and Richardson-Lucy.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

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
    int nparts = 0;
    IterState* st = nullptr;
    double* f_hist = nullptr;
    double* d_hist = nullptr;
    GradPsfPlan gp{};
    double* gp_part = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    struct Key {
        const float* y;
        float* x;
        int K;
        int policy, max_halvings, max_rejects;
        double delta0, beta;
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
        for (void* v : allocs) cudaFree(v);
        allocs.clear();
        if (cap) cudaStreamDestroy(cap);
        cap = nullptr;
    }
};

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

cdv_status cdv_plan_create(cdv_plan** out, int n, const int64_t* m, const int32_t* p, cdv_mode mode, void* stream)
{
    (void)stream;
    if (!out) return fail(CDV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!m || !p) return fail(CDV_ERR_INVALID_ARG, "m or p is NULL");
    if (n < 1 || n > 3) return fail(CDV_ERR_SHAPE, "n = %d, must be 1, 2 or 3", n);
    if (mode != CDV_MODE_FP32 && mode != CDV_MODE_BF16 && mode != CDV_MODE_TF32 && mode != CDV_MODE_SPLIT_BF16X3)
        return fail(CDV_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
    if (mode != CDV_MODE_FP32) return fail(CDV_ERR_UNSUPPORTED, "mode %d has no kernel in this build", (int)mode);
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
    if (!conv_fp32_supported(P->q[2])) {
        delete P;
        return fail(CDV_ERR_UNSUPPORTED, "template width %d along the contiguous axis: this build supports odd 1..31",
                    P->q[2]);
    }
    P->gf = ConvGeom{P->m[0], P->m[1], P->m[2],
                     P->m[0] + 2 * P->p[0], P->m[1] + 2 * P->p[1], P->m[2] + 2 * P->p[2],
                     0, 0, 0, P->q[0], P->q[1], P->q[2]};
    P->ga = ConvGeom{P->gf.b1, P->gf.b2, P->gf.b3, P->m[0], P->m[1], P->m[2],
                     2 * P->p[0], 2 * P->p[1], 2 * P->p[2], P->q[0], P->q[1], P->q[2]};
    P->tf = conv_fp32_tile(P->gf);
    P->ta = conv_fp32_tile(P->ga);
    P->nparts = std::max(P->tf.grid, P->ta.grid);
    P->gp = GradPsfPlan{P->m[0], P->m[1], P->m[2], P->q[0], P->q[1], P->q[2], 1,
                        std::max(1, (152 * 4 + P->q[0] - 1) / P->q[0])};

    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess) e = conv_fp32_prepare(P->q[2]);
    if (e == cudaSuccess) e = grad_psf_prepare();
    if (e == cudaSuccess && small_supported(P->m, P->p)) {
        SmallRun r{};
        for (int i = 0; i < 3; i++) {
            r.m[i] = P->m[i];
            r.p[i] = P->p[i];
        }
        e = small_iterate(r, nullptr, true);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking);
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
    cudaStream_t s = (cudaStream_t)stream;
    CDV_CUDA(cudaMemcpyAsync(plan->H, H, plan->nh * sizeof(float), cudaMemcpyDeviceToDevice, s), "copy H");
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
    c.st = P->st;
    c.f_hist = P->f_hist;
    c.d_hist = P->d_hist;
    return c;
}

static cdv_status enqueue_run(cdv_plan* P, const float* Y, float* X, int K, const cdv_iter_opts& o, cudaStream_t s)
{
    const IterCtx c = make_ctx(P, Y, X);
    CDV_CUDA(launch_x0(o.x0_policy, X, Y, P->m[0], P->m[1], P->m[2], P->p[0], P->p[1], P->p[2], s), "x0");
    CDV_CUDA(launch_state_init(P->st, o.delta0, P->absum, o.beta, o.max_halvings, o.max_rejects, K, kHistCap, s), "state");
    ConvLaunch F{};
    F.g = P->gf;
    F.w = P->H;
    F.batch = 1;
    F.ctx = c;
    ConvLaunch A = F;
    A.g = P->ga;
    A.w = P->Ht;
    F.role = ROLE_FWD_INIT;
    CDV_CUDA(conv_fp32_launch(F, P->tf, s), "forward (initial)");
    CDV_CUDA(launch_decide(c, P->tf.grid, 0, 1, s), "decide (initial)");
    F.role = ROLE_FWD_TRIAL;
    A.role = ROLE_ADJ_TRIAL;
    const int slots = K + o.max_rejects;
    for (int i = 0; i < slots && K > 0; i++) {
        CDV_CUDA(conv_fp32_launch(A, P->ta, s), "adjoint trial");
        CDV_CUDA(conv_fp32_launch(F, P->tf, s), "forward trial");
        CDV_CUDA(launch_decide(c, P->tf.grid, P->ta.grid, 0, s), "decide");
    }
    CDV_CUDA(launch_finalize(c, P->nx, s), "finalize");
    return CDV_OK;
}

static cdv_status fill_report(cdv_plan* P, int K, cdv_iter_report* rep, cudaStream_t s)
{
    CDV_CUDA(cudaStreamSynchronize(s), "iterate sync");
    IterState st;
    CDV_CUDA(cudaMemcpy(&st, P->st, sizeof st, cudaMemcpyDeviceToHost), "read state");
    rep->accepted = st.accepted;
    rep->rejected = st.rejected;
    rep->status = st.status;
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
    if (o.path < CDV_PATH_AUTO || o.path > CDV_PATH_SMALL) return fail(CDV_ERR_INVALID_ARG, "path = %d", o.path);
    const double delta0 = o.delta0 > 0.0 ? o.delta0 : 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    const bool small_ok = small_supported(plan->m, plan->p);
    if (o.path == CDV_PATH_SMALL && !small_ok)
        return fail(CDV_ERR_UNSUPPORTED, "problem does not fit the single-CTA path (%zu bytes of shared memory)",
                    small_smem_bytes(plan->m, plan->p));
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
        cdv_plan::Key k{Y, X, K, o.x0_policy, o.max_halvings, o.max_rejects, delta0, o.beta};
        const bool same = plan->key_valid && memcmp(&k, &plan->key, sizeof k) == 0;
        if (!same) {
            if (plan->gexec) cudaGraphExecDestroy(plan->gexec);
            if (plan->graph) cudaGraphDestroy(plan->graph);
            plan->gexec = nullptr;
            plan->graph = nullptr;
            plan->key_valid = false;
            CDV_CUDA(cudaStreamBeginCapture(plan->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
            cdv_status st = enqueue_run(plan, Y, X, K, o, plan->cap);
            cudaGraph_t gr = nullptr;
            cudaError_t e = cudaStreamEndCapture(plan->cap, &gr);
            if (st != CDV_OK) {
                if (gr) cudaGraphDestroy(gr);
                return st;
            }
            if (e != cudaSuccess) return cuda_fail(e, "end capture");
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

cdv_status cdv_plan_sync_status(cdv_plan* plan, void* stream)
{
    if (!plan) return fail(CDV_ERR_INVALID_ARG, "plan is NULL");
    CDV_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "sync");
    CDV_CUDA(cudaGetLastError(), "pending error");
    return CDV_OK;
}

}  // extern "C"

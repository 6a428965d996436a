// Batched solver: many independent volumes, each with its own size and
// template, iterated together (Steps 1-3 applied to every volume).
//
// By default (CDV_PATH_AUTO or CDV_PATH_PERSISTENT) one persistent launch runs
// the whole K-step run of every volume (conv_fp32_persist.cu): its CTAs take
// tiles of any volume whose current phase has tiles left, and the CTA that
// completes a phase runs that volume's step rule, so each volume advances at
// its own pace.  With CDV_PATH_GENERAL all volumes advance in lockstep through
// the same trial slots instead; one slot is one batched adjoint launch and one
// batched forward launch per template width present (each CTA of such a launch
// computes one tile of one volume, chosen from a work list ordered largest
// volume first), plus one batched decision launch (one block per volume, each
// with its own FP64 step rule), and the K-step run is a WHILE loop over trial
// slots that ends when every volume is done.  Either run is one CUDA graph,
// captured once and replayed.  Per-volume tile
// shapes come from a timing autotuner whose results are cached per process
// (keyed by device, geometry and direction); the arithmetic of every output
// sample does not depend on the tile shape, so a volume's iterates are
// identical to those of cdv_iterate on that volume alone.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cdv_internal.h"

using namespace cdv;

namespace {

cdv_status bfail(cdv_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return s;
}

#define BCUDA(call, what)                                                                                   \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) return bfail(CDV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e_));         \
    } while (0)

constexpr int kBatchHist = 4096;

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;     // geometry key -> chosen thread rows

std::string tune_key(int dev, const ConvGeom& g)
{
    char b[256];
    snprintf(b, sizeof b, "%d|%lld,%lld,%lld|%lld,%lld,%lld|%d,%d,%d|%d,%d,%d", dev, (long long)g.a1, (long long)g.a2,
             (long long)g.a3, (long long)g.b1, (long long)g.b2, (long long)g.b3, g.o1, g.o2, g.o3, g.q1, g.q2, g.q3);
    return b;
}

}  // namespace

struct cdv_batch {
    struct Vol {
        int64_t m[3] = {1, 1, 1};
        int p[3] = {0, 0, 0}, q[3] = {1, 1, 1};
        int64_t nx = 0, ny = 0, nh = 0;
        ConvGeom gf{}, ga{};
        ConvTile tf{}, ta{};
        float *H = nullptr, *Ht = nullptr, *xw = nullptr, *r0 = nullptr, *r1 = nullptr, *g = nullptr;
        double *absum = nullptr, *part_f = nullptr, *part_m = nullptr, *f_hist = nullptr, *d_hist = nullptr;
        IterState* st = nullptr;
    };
    struct Group {
        int q3;
        int off_f, n_f, off_a, n_a;
        size_t smem_f, smem_a;
    };
    int count = 0, n = 0, device = 0;
    std::vector<Vol> v;
    std::vector<Group> groups;
    std::vector<void*> allocs;
    size_t bytes = 0;
    bool has_psf = false;
    ConvBatchVol* d_fwd_init = nullptr;
    ConvBatchVol* d_fwd_trial = nullptr;
    ConvBatchVol* d_adj_trial = nullptr;
    BatchVolCtx* d_ctx = nullptr;
    int2* d_items_f = nullptr;
    int2* d_items_a = nullptr;
    // persistent run: scan order, per-volume phase words and tile counters, retired count, error word
    int* d_order = nullptr;
    int2* d_ntiles = nullptr;
    unsigned long long* d_word = nullptr;
    int* d_tiles_done = nullptr;
    int* d_flags = nullptr;             // [0] volumes retired, [1] error
    size_t psmem = 0;
    int pgrid = 0;
    long long wait_cycles = kTcWaitCycles;
    cudaStream_t cap = nullptr;
    // one stream per template-width group: the groups' launches of a trial slot run side by side
    // (captured as parallel graph branches), joined before the decision
    std::vector<cudaStream_t> gstream;
    std::vector<cudaEvent_t> gdone;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<const float*> key_y;
    std::vector<float*> key_x;
    int key_K = -1;
    int key_persist = -1;
    cdv_iter_opts key_o{};
    bool key_valid = false;

    template <class T>
    cudaError_t alloc(T** ptr, size_t count_)
    {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(count_, 1) * sizeof(T));
        if (e != cudaSuccess) return e;
        allocs.push_back(p);
        bytes += count_ * sizeof(T);
        *ptr = static_cast<T*>(p);
        return cudaSuccess;
    }
    void release()
    {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
        for (void* p : allocs) cudaFree(p);
        allocs.clear();
        if (cap) cudaStreamDestroy(cap);
        cap = nullptr;
        for (cudaStream_t t : gstream) cudaStreamDestroy(t);
        gstream.clear();
        for (cudaEvent_t t : gdone) cudaEventDestroy(t);
        gdone.clear();
        if (fork) cudaEventDestroy(fork);
        fork = nullptr;
    }
};

// Time one plain launch of the FP32 engine for each candidate row count and keep the fastest.
static int autotune_rows(int dev, const ConvGeom& g, const float* in, float* out, const float* w, cudaStream_t s)
{
    const std::string key = tune_key(dev, g);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) return it->second;
    }
    const ConvTile def = conv_fp32_tile(g);
    std::vector<int> cand = {def.nty};
    for (int c : {2, 4, 8, 16, 32}) {
        const ConvTile t = conv_fp32_tile_shape(g, c);
        if (std::find(cand.begin(), cand.end(), t.nty) == cand.end() && t.smem <= 110 * 1024) cand.push_back(t.nty);
    }
    int best = def.nty;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return best;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return best;
    }
    for (int c : cand) {
        const ConvTile t = conv_fp32_tile_shape(g, c);
        ConvLaunch L{};
        L.g = g;
        L.in = in;
        L.out = out;
        L.w = w;
        L.role = ROLE_PLAIN;
        L.batch = 1;
        if (conv_fp32_launch(L, t, s) != cudaSuccess) continue;     // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < 2; r++) conv_fp32_launch(L, t, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = t.nty;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
    return best;
}

extern "C" {

cdv_status cdv_batch_plan_create(cdv_batch** out, int count, int n, const int64_t* m, const int32_t* p, cdv_mode mode,
                                 int autotune, void* stream)
{
    if (!out) return bfail(CDV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!m || !p || count < 1) return bfail(CDV_ERR_INVALID_ARG, "count = %d or NULL sizes", count);
    if (n < 1 || n > 3) return bfail(CDV_ERR_SHAPE, "n = %d, must be 1, 2 or 3", n);
    if (mode != CDV_MODE_FP32) return bfail(CDV_ERR_UNSUPPORTED, "the batched solver runs in CDV_MODE_FP32");
    cdv_batch* B = new cdv_batch();
    B->count = count;
    B->n = n;
    B->v.resize(count);
    cudaError_t e = cudaGetDevice(&B->device);
    for (int i = 0; i < count && e == cudaSuccess; i++) {
        cdv_batch::Vol& V = B->v[i];
        for (int a = 0; a < n; a++) {
            const int64_t mm = m[(size_t)i * n + a];
            const int pp = p[(size_t)i * n + a];
            if (mm < 1 || pp < 0 || mm > (1LL << 31) || pp > (1 << 20)) {
                B->release();
                delete B;
                return bfail(CDV_ERR_SHAPE, "volume %d axis %d: m = %lld, p = %d", i, a, (long long)mm, pp);
            }
            V.m[3 - n + a] = mm;
            V.p[3 - n + a] = pp;
        }
        for (int a = 0; a < 3; a++) V.q[a] = 2 * V.p[a] + 1;
        if (!conv_fp32_supported(V.q[2])) {
            B->release();
            delete B;
            return bfail(CDV_ERR_UNSUPPORTED, "volume %d: template width %d along the contiguous axis", i, V.q[2]);
        }
        V.nx = V.m[0] * V.m[1] * V.m[2];
        V.ny = (V.m[0] + 2 * V.p[0]) * (V.m[1] + 2 * V.p[1]) * (V.m[2] + 2 * V.p[2]);
        V.nh = (int64_t)V.q[0] * V.q[1] * V.q[2];
        V.gf = ConvGeom{V.m[0], V.m[1], V.m[2], V.m[0] + 2 * V.p[0], V.m[1] + 2 * V.p[1], V.m[2] + 2 * V.p[2],
                        0, 0, 0, V.q[0], V.q[1], V.q[2]};
        V.ga = ConvGeom{V.gf.b1, V.gf.b2, V.gf.b3, V.m[0], V.m[1], V.m[2], 2 * V.p[0], 2 * V.p[1], 2 * V.p[2],
                        V.q[0], V.q[1], V.q[2]};
        V.tf = conv_fp32_tile(V.gf);
        V.ta = conv_fp32_tile(V.ga);
        // partials: one per CTA for any tile shape the autotuner may pick (at least one thread row per CTA)
        const int64_t nparts = std::max(conv_fp32_tile_shape(V.gf, 1).grid, conv_fp32_tile_shape(V.ga, 1).grid);
        if (e == cudaSuccess) e = B->alloc(&V.H, V.nh);
        if (e == cudaSuccess) e = B->alloc(&V.Ht, V.nh);
        if (e == cudaSuccess) e = B->alloc(&V.absum, 1);
        if (e == cudaSuccess) e = B->alloc(&V.xw, V.nx);
        if (e == cudaSuccess) e = B->alloc(&V.g, V.nx);
        if (e == cudaSuccess) e = B->alloc(&V.r0, V.ny);
        if (e == cudaSuccess) e = B->alloc(&V.r1, V.ny);
        if (e == cudaSuccess) e = B->alloc(&V.part_f, (size_t)nparts);
        if (e == cudaSuccess) e = B->alloc(&V.part_m, (size_t)nparts);
        if (e == cudaSuccess) e = B->alloc(&V.st, 1);
        if (e == cudaSuccess) e = B->alloc(&V.f_hist, kBatchHist + 1);
        if (e == cudaSuccess) e = B->alloc(&V.d_hist, kBatchHist);
    }
    if (e == cudaSuccess) e = B->alloc(&B->d_fwd_init, count);
    if (e == cudaSuccess) e = B->alloc(&B->d_fwd_trial, count);
    if (e == cudaSuccess) e = B->alloc(&B->d_adj_trial, count);
    if (e == cudaSuccess) e = B->alloc(&B->d_ctx, count);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    for (int i = 0; i < count && e == cudaSuccess; i++) e = conv_fp32_prepare(B->v[i].q[2]);
    for (int i = 0; i < count && e == cudaSuccess; i++) e = conv_fp32_batch_launch(B->v[i].q[2], nullptr, nullptr, 0, 0, nullptr);
    // tile shapes: autotuned (timed on zeroed workspace with a zero template) or the default
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < count && e == cudaSuccess; i++) {
        cdv_batch::Vol& V = B->v[i];
        if (autotune) {
            e = cudaMemsetAsync(V.xw, 0, V.nx * sizeof(float), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(V.r0, 0, V.ny * sizeof(float), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(V.H, 0, V.nh * sizeof(float), s);
            if (e != cudaSuccess) break;
            V.tf = conv_fp32_tile_shape(V.gf, autotune_rows(B->device, V.gf, V.xw, V.r0, V.H, s));
            V.ta = conv_fp32_tile_shape(V.ga, autotune_rows(B->device, V.ga, V.r0, V.g, V.H, s));
        }
    }
    // work lists: per template width, (volume, tile) items, largest volume first
    std::vector<int> order(count);
    for (int i = 0; i < count; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        return B->v[a].nx * B->v[a].nh > B->v[b].nx * B->v[b].nh;
    });
    std::vector<int2> items_f, items_a;
    for (int q3 = 1; q3 <= 31; q3 += 2) {
        cdv_batch::Group gr{q3, (int)items_f.size(), 0, (int)items_a.size(), 0, 0, 0};
        for (int i : order) {
            const cdv_batch::Vol& V = B->v[i];
            if (V.q[2] != q3) continue;
            for (int t = 0; t < V.tf.grid; t++) items_f.push_back(make_int2(i, t));
            for (int t = 0; t < V.ta.grid; t++) items_a.push_back(make_int2(i, t));
            gr.smem_f = std::max(gr.smem_f, V.tf.smem);
            gr.smem_a = std::max(gr.smem_a, V.ta.smem);
        }
        gr.n_f = (int)items_f.size() - gr.off_f;
        gr.n_a = (int)items_a.size() - gr.off_a;
        if (gr.n_f > 0) B->groups.push_back(gr);
    }
    for (size_t i = 0; e == cudaSuccess && i < B->groups.size(); i++) {
        cudaStream_t t = nullptr;
        cudaEvent_t d = nullptr;
        e = cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking);
        if (e == cudaSuccess) B->gstream.push_back(t);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d, cudaEventDisableTiming);
        if (e == cudaSuccess) B->gdone.push_back(d);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    // persistent run: volumes scanned in the work lists' order, shared memory for any tile of the batch
    if (e == cudaSuccess) e = B->alloc(&B->d_order, count);
    if (e == cudaSuccess) e = B->alloc(&B->d_word, count);
    if (e == cudaSuccess) e = B->alloc(&B->d_tiles_done, count);
    if (e == cudaSuccess) e = B->alloc(&B->d_flags, 2);
    if (e == cudaSuccess) e = cudaMemcpy(B->d_order, order.data(), count * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = B->alloc(&B->d_ntiles, count);
    if (e == cudaSuccess) {
        std::vector<int2> nt(count);
        for (int k = 0; k < count; k++) nt[k] = make_int2(B->v[order[k]].tf.grid, B->v[order[k]].ta.grid);
        e = cudaMemcpy(B->d_ntiles, nt.data(), count * sizeof(int2), cudaMemcpyHostToDevice);
    }
    B->psmem = 512 * sizeof(double);
    for (int i = 0; i < count; i++) B->psmem = std::max(B->psmem, std::max(B->v[i].tf.smem, B->v[i].ta.smem));
    if (e == cudaSuccess) e = conv_fp32_persist_prepare();
    if (e == cudaSuccess) {
        B->pgrid = conv_fp32_persist_grid(B->psmem);
        if (B->pgrid < 1) e = cudaErrorInvalidConfiguration;
    }
    if (e == cudaSuccess) e = B->alloc(&B->d_items_f, items_f.size());
    if (e == cudaSuccess) e = B->alloc(&B->d_items_a, items_a.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(B->d_items_f, items_f.data(), items_f.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(B->d_items_a, items_a.data(), items_a.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        cudaGetLastError();
        B->release();
        delete B;
        return oom ? bfail(CDV_ERR_OOM, "batch workspace allocation failed")
                   : bfail(CDV_ERR_CUDA, "batch plan create: %s", cudaGetErrorString(e));
    }
    *out = B;
    return CDV_OK;
}

cdv_status cdv_batch_workspace_size(const cdv_batch* b, size_t* bytes)
{
    if (!b || !bytes) return bfail(CDV_ERR_INVALID_ARG, "NULL argument");
    *bytes = b->bytes;
    return CDV_OK;
}

cdv_status cdv_batch_set_psfs(cdv_batch* b, const float* const* H, void* stream)
{
    if (!b || !H) return bfail(CDV_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < b->count; i++) {
        cdv_batch::Vol& V = b->v[i];
        if (!H[i]) return bfail(CDV_ERR_INVALID_ARG, "template %d is NULL", i);
        BCUDA(cudaMemcpyAsync(V.H, H[i], V.nh * sizeof(float), cudaMemcpyDeviceToDevice, s), "copy H");
        BCUDA(launch_flip(V.H, V.Ht, V.q[0], V.q[1], V.q[2], s), "flip H");
        BCUDA(launch_abs_sum(V.H, V.nh, V.absum, s), "sum |H|");
    }
    b->has_psf = true;
    return CDV_OK;
}

static cdv_status batch_tables(cdv_batch* b, const float* const* Y, float* const* X)
{
    std::vector<ConvBatchVol> fi(b->count), ft(b->count), at(b->count);
    std::vector<BatchVolCtx> cx(b->count);
    for (int i = 0; i < b->count; i++) {
        cdv_batch::Vol& V = b->v[i];
        IterCtx c{};
        c.x[0] = X[i];
        c.x[1] = V.xw;
        c.r[0] = V.r0;
        c.r[1] = V.r1;
        c.g = V.g;
        c.y = Y[i];
        c.part_f = V.part_f;
        c.part_m = V.part_m;
        c.st = V.st;
        c.f_hist = V.f_hist;
        c.d_hist = V.d_hist;
        ConvLaunch F{};
        F.g = V.gf;
        F.w = V.H;
        F.batch = 1;
        F.ctx = c;
        F.role = ROLE_FWD_INIT;
        fi[i] = ConvBatchVol{F, V.tf.ntx, V.tf.nty, V.tf.tiles2, V.tf.tiles3, V.tf.smem};
        F.role = ROLE_FWD_TRIAL;
        ft[i] = ConvBatchVol{F, V.tf.ntx, V.tf.nty, V.tf.tiles2, V.tf.tiles3, V.tf.smem};
        ConvLaunch A = F;
        A.g = V.ga;
        A.w = V.Ht;
        A.role = ROLE_ADJ_TRIAL;
        at[i] = ConvBatchVol{A, V.ta.ntx, V.ta.nty, V.ta.tiles2, V.ta.tiles3, V.ta.smem};
        cx[i] = BatchVolCtx{c, V.m[0], V.m[1], V.m[2], V.p[0], V.p[1], V.p[2], V.tf.grid, V.ta.grid, V.absum};
    }
    BCUDA(cudaMemcpy(b->d_fwd_init, fi.data(), fi.size() * sizeof(ConvBatchVol), cudaMemcpyHostToDevice), "tables");
    BCUDA(cudaMemcpy(b->d_fwd_trial, ft.data(), ft.size() * sizeof(ConvBatchVol), cudaMemcpyHostToDevice), "tables");
    BCUDA(cudaMemcpy(b->d_adj_trial, at.data(), at.size() * sizeof(ConvBatchVol), cudaMemcpyHostToDevice), "tables");
    BCUDA(cudaMemcpy(b->d_ctx, cx.data(), cx.size() * sizeof(BatchVolCtx), cudaMemcpyHostToDevice), "tables");
    return CDV_OK;
}

struct BatchRun {
    cdv_batch* b;
    int K;
    cdv_iter_opts o;
};

// The convolutions of one slot: per template-width group (its own stream, forked from s) the adjoint
// trial then the forward trial (trial), or the initial forward (prologue); all groups joined back
// into s.  A volume belongs to one group, so its adjoint precedes its forward; groups are independent.
static cdv_status batch_groups(cdv_batch* b, bool trial, cudaStream_t s)
{
    BCUDA(cudaEventRecord(b->fork, s), "fork");
    for (size_t i = 0; i < b->groups.size(); i++) {
        const auto& g = b->groups[i];
        cudaStream_t t = b->gstream[i];
        BCUDA(cudaStreamWaitEvent(t, b->fork, 0), "fork wait");
        if (trial) {
            BCUDA(conv_fp32_batch_launch(g.q3, b->d_adj_trial, b->d_items_a + g.off_a, g.n_a, g.smem_a, t), "adjoint");
            BCUDA(conv_fp32_batch_launch(g.q3, b->d_fwd_trial, b->d_items_f + g.off_f, g.n_f, g.smem_f, t), "forward");
        } else {
            BCUDA(conv_fp32_batch_launch(g.q3, b->d_fwd_init, b->d_items_f + g.off_f, g.n_f, g.smem_f, t), "forward");
        }
        BCUDA(cudaEventRecord(b->gdone[i], t), "join");
        BCUDA(cudaStreamWaitEvent(s, b->gdone[i], 0), "join wait");
    }
    return CDV_OK;
}

// Phases of a batched run (see build_loop_graph): 0 prologue, 1 one trial slot for every volume,
// 2 epilogue.  In a loop graph the slot ends with the loop condition (any volume still running).
static cdv_status batch_phase(void* vctx, int phase, bool loop, unsigned long long h, cudaStream_t s)
{
    BatchRun& R = *static_cast<BatchRun*>(vctx);
    cdv_batch* b = R.b;
    const int max_trials = R.K + R.o.max_rejects + 1;
    if (phase == 0) {
        BCUDA(launch_batch_x0(b->d_ctx, b->count, R.o.x0_policy, s), "x0");
        BCUDA(launch_batch_state_init(b->d_ctx, b->count, R.o.delta0 > 0.0 ? R.o.delta0 : 0.0, R.o.beta,
                                      R.o.max_halvings, R.o.max_rejects, R.K, kBatchHist, s), "state");
        cdv_status st = batch_groups(b, false, s);
        if (st != CDV_OK) return st;
        BCUDA(launch_batch_decide(b->d_ctx, b->count, 1, s), "decide");
    } else if (phase == 1) {
        cdv_status st = batch_groups(b, true, s);
        if (st != CDV_OK) return st;
        BCUDA(launch_batch_decide(b->d_ctx, b->count, 0, s), "decide");
    } else {
        BCUDA(launch_batch_finalize(b->d_ctx, b->count, s), "finalize");
        return CDV_OK;
    }
    if (loop) BCUDA(launch_batch_loop_cond(b->d_ctx, b->count, h, max_trials, s), "loop condition");
    return CDV_OK;
}

// The persistent run: reset the phase words and counters, x0 and the states, one launch for every
// volume's whole run, then x_K into the caller's arrays.
static cdv_status batch_persist_enqueue(cdv_batch* b, int K, const cdv_iter_opts& o, cudaStream_t s)
{
    BCUDA(cudaMemsetAsync(b->d_word, 0, b->count * sizeof(unsigned long long), s), "reset phases");
    BCUDA(cudaMemsetAsync(b->d_tiles_done, 0, b->count * sizeof(int), s), "reset counters");
    BCUDA(cudaMemsetAsync(b->d_flags, 0, 2 * sizeof(int), s), "reset flags");
    BCUDA(launch_batch_x0(b->d_ctx, b->count, o.x0_policy, s), "x0");
    BCUDA(launch_batch_state_init(b->d_ctx, b->count, o.delta0 > 0.0 ? o.delta0 : 0.0, o.beta, o.max_halvings,
                                  o.max_rejects, K, kBatchHist, s), "state");
    BatchPersist P{b->d_fwd_init, b->d_fwd_trial, b->d_adj_trial, b->d_ctx, b->d_order, b->d_ntiles, b->d_word, b->d_tiles_done,
                   b->d_flags, b->d_flags + 1, b->count, K + o.max_rejects + 1, b->wait_cycles};
    BCUDA(conv_fp32_persist_launch(P, b->pgrid, b->psmem, s), "persistent run");
    BCUDA(launch_batch_finalize(b->d_ctx, b->count, s), "finalize");
    return CDV_OK;
}

static cdv_status batch_enqueue(cdv_batch* b, int K, const cdv_iter_opts& o, cudaStream_t s)
{
    BatchRun R{b, K, o};
    cdv_status st = batch_phase(&R, 0, false, 0, s);
    for (int i = 0; st == CDV_OK && K > 0 && i < K + o.max_rejects; i++) st = batch_phase(&R, 1, false, 0, s);
    if (st == CDV_OK) st = batch_phase(&R, 2, false, 0, s);
    return st;
}

cdv_status cdv_batch_iterate(cdv_batch* b, const float* const* Y, float* const* X, int K, const cdv_iter_opts* opts,
                             cdv_iter_report* reports, void* stream)
{
    if (!b || !Y || !X) return bfail(CDV_ERR_INVALID_ARG, "NULL argument");
    if (K < 0 || K > kBatchHist) return bfail(CDV_ERR_INVALID_ARG, "K = %d (0..%d)", K, kBatchHist);
    if (!b->has_psf) return bfail(CDV_ERR_NO_PSF, "no templates set");
    for (int i = 0; i < b->count; i++)
        if (!Y[i] || !X[i]) return bfail(CDV_ERR_INVALID_ARG, "volume %d: NULL array", i);
    cdv_iter_opts o;
    if (opts) o = *opts; else cdv_iter_opts_default(&o);
    if (o.x0_policy < CDV_X0_GIVEN || o.x0_policy > CDV_X0_ZERO || !(o.beta > 0.0 && o.beta < 1.0) ||
        o.max_halvings < 0 || o.max_rejects < 0 || o.max_rejects > (1 << 20))
        return bfail(CDV_ERR_INVALID_ARG, "iteration options");
    if (o.tikhonov != 0.0 || o.armijo != 0.0 || o.bb != 0)
        return bfail(CDV_ERR_UNSUPPORTED, "the batched solver runs the plain step rule (tikhonov = armijo = bb = 0)");
    if (o.path == CDV_PATH_SMALL || o.path < CDV_PATH_AUTO || o.path > CDV_PATH_PERSISTENT)
        return bfail(o.path == CDV_PATH_SMALL ? CDV_ERR_UNSUPPORTED : CDV_ERR_INVALID_ARG,
                     "path = %d: the batched solver runs CDV_PATH_PERSISTENT (AUTO) or CDV_PATH_GENERAL", o.path);
    const int persist = o.path != CDV_PATH_GENERAL;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<const float*> ky(Y, Y + b->count);
    std::vector<float*> kx(X, X + b->count);
    const bool same = b->key_valid && ky == b->key_y && kx == b->key_x && K == b->key_K &&
                      persist == b->key_persist && memcmp(&o, &b->key_o, sizeof o) == 0;
    if (!same || !o.use_graph) {
        BCUDA(cudaStreamSynchronize(s), "sync before table update");
        cdv_status st = batch_tables(b, Y, X);
        if (st != CDV_OK) return st;
    }
    if (o.use_graph) {
        if (!same) {
            if (b->gexec) cudaGraphExecDestroy(b->gexec);
            if (b->graph) cudaGraphDestroy(b->graph);
            b->gexec = nullptr;
            b->graph = nullptr;
            b->key_valid = false;
            BatchRun R{b, K, o};
            cudaGraph_t gr = nullptr;
            cdv_status st = CDV_OK;
            if (persist) {
                BCUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
                st = batch_persist_enqueue(b, K, o, b->cap);
                cudaGraph_t tmp = nullptr;
                const cudaError_t e2 = cudaStreamEndCapture(b->cap, &tmp);
                if (st != CDV_OK) {
                    if (tmp) cudaGraphDestroy(tmp);
                    return st;
                }
                BCUDA(e2, "end capture");
                gr = tmp;
            } else {
                st = build_loop_graph(b->cap, batch_phase, &R, &gr);
            }
            if (st != CDV_OK) return st;
            b->graph = gr;
            BCUDA(cudaGraphInstantiate(&b->gexec, gr, 0), "instantiate graph");
            b->key_y = ky;
            b->key_x = kx;
            b->key_K = K;
            b->key_persist = persist;
            b->key_o = o;
            b->key_valid = true;
        }
        BCUDA(cudaGraphLaunch(b->gexec, s), "graph launch");
    } else {
        b->key_valid = false;
        cdv_status st = persist ? batch_persist_enqueue(b, K, o, s) : batch_enqueue(b, K, o, s);
        if (st != CDV_OK) return st;
    }
    if (!reports) return CDV_OK;
    BCUDA(cudaStreamSynchronize(s), "batch sync");
    if (persist) {
        int flags[2] = {0, 0};
        BCUDA(cudaMemcpy(flags, b->d_flags, sizeof flags, cudaMemcpyDeviceToHost), "read flags");
        if (flags[1]) return bfail(CDV_ERR_TIMEOUT, "persistent batched run: a CTA found no tile within the wait budget");
    }
    for (int i = 0; i < b->count; i++) {
        const cdv_batch::Vol& V = b->v[i];
        IterState st;
        BCUDA(cudaMemcpy(&st, V.st, sizeof st, cudaMemcpyDeviceToHost), "read state");
        cdv_iter_report& r = reports[i];
        r.accepted = st.accepted;
        r.rejected = st.rejected;
        r.status = st.status;
        r.trials = st.trials;
        double f0 = 0.0;
        BCUDA(cudaMemcpy(&f0, V.f_hist, sizeof(double), cudaMemcpyDeviceToHost), "read f0");
        r.f0 = f0;
        r.f_final = st.f_cur;
        r.gmac = (double)(1 + st.trials + st.adj_convs) * (double)V.nx * (double)V.nh * 1e-9;
        const int nh = std::min(st.accepted, K);
        if (r.f_hist)
            BCUDA(cudaMemcpy(r.f_hist, V.f_hist, (nh + 1) * sizeof(double), cudaMemcpyDeviceToHost), "read f");
        if (r.delta_hist && nh > 0)
            BCUDA(cudaMemcpy(r.delta_hist, V.d_hist, nh * sizeof(double), cudaMemcpyDeviceToHost), "read delta");
    }
    return CDV_OK;
}

cdv_status cdv_batch_set_wait_cycles(cdv_batch* b, long long cycles)
{
    if (!b) return bfail(CDV_ERR_INVALID_ARG, "NULL batch plan");
    if (cycles < 0) return bfail(CDV_ERR_INVALID_ARG, "cycles = %lld", cycles);
    b->wait_cycles = cycles == 0 ? kTcWaitCycles : cycles;
    b->key_valid = false;                  // a captured graph holds the old launch parameters
    return CDV_OK;
}

cdv_status cdv_batch_destroy(cdv_batch* b)
{
    if (!b) return CDV_OK;
    b->release();
    delete b;
    return CDV_OK;
}

}  // extern "C"

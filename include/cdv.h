/*
 * cdv -- direct-convolution deconvolution on GB300 (sm_103a).
 *
 * C ABI of the hot path of "Properties on n-dimensional convolution for image
 * deconvolution" (arXiv 1711.11224): the full n-D convolution Y = X (*) H
 * (Property 1, Eq. 1), its adjoint (A_n^h)^T R = M_2p(R (*) H~) (Property 2,
 * Eq. 2), and the projected-gradient non-negative least-squares iteration
 * built from the two (Steps 1-3 and Eq. 6 of the 2-D application, applied to
 * n = 1, 2, 3).
 *
 * Notation follows the paper: X has m_i samples per axis, the template H has
 * q_i = 2 p_i + 1, Y and every residual R have m_i + 2 p_i.  Arrays are dense
 * C-order float32 (axis 1 slowest, axis n contiguous: the row partition of the
 * vectorisation X^v), in DEVICE memory unless a name ends in _host.
 *
 * Conventions for every call:
 *  - The caller owns every array it passes; the library never frees them.
 *    A plan owns its copy of H, the flipped template and a workspace, all
 *    allocated by cdv_plan_create / cdv_plan_set_psf and freed by
 *    cdv_plan_destroy.  cdv_forward, cdv_adjoint and cdv_iterate allocate
 *    nothing.
 *  - `stream` is a cudaStream_t passed as void* (NULL: the legacy default
 *    stream).  Work is enqueued asynchronously on it unless a call says it
 *    synchronises.
 *  - Argument errors return before anything is enqueued.  CUDA launch errors
 *    return CDV_ERR_CUDA.  Errors raised on the device (non-finite values, a
 *    wait that timed out) are recorded in the plan's device status word and
 *    returned by cdv_plan_sync_status.
 *  - A plan is not thread-safe: one host thread at a time per plan.
 *  - There is no CPU fallback: without a usable CUDA device every call that
 *    computes returns CDV_ERR_CUDA.
 */
#ifndef CDV_H
#define CDV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CDV_OK = 0,
    CDV_ERR_INVALID_ARG = 1,    /* null pointer, bad enum, K < 0, ... */
    CDV_ERR_SHAPE = 2,          /* n not in {1,2,3}, m_i < 1, p_i < 0, sizes overflow */
    CDV_ERR_UNSUPPORTED = 3,    /* a size or mode this build has no kernel for */
    CDV_ERR_OOM = 4,            /* workspace allocation failed */
    CDV_ERR_CUDA = 5,           /* a CUDA runtime call failed */
    CDV_ERR_TIMEOUT = 6,        /* a bounded device-side wait ran out */
    CDV_ERR_NOT_DESCENDING = 7, /* the step rule found no decreasing step */
    CDV_ERR_NONFINITE = 8,      /* NaN/Inf met in the objective */
    CDV_ERR_NO_PSF = 9          /* cdv_plan_set_psf was not called */
} cdv_status;

/* Arithmetic of the two convolutions (the iteration's scalars are FP64 in
 * every mode). */
typedef enum {
    CDV_MODE_FP32 = 0,          /* FP32 FMA on CUDA cores */
    CDV_MODE_BF16 = 1,          /* tensor cores, BF16 products, FP32 accumulate */
    CDV_MODE_TF32 = 2,          /* tensor cores, TF32 products, FP32 accumulate */
    CDV_MODE_SPLIT_BF16X3 = 3,  /* tensor cores, x_hi h_hi + x_hi h_lo + x_lo h_hi */
    CDV_MODE_FFT = 4,           /* comparator, not the paper's method: both operators through FP32
                                   cuFFT transforms of a zero-padded grid (the FFT approach the
                                   paper's introduction contrasts with); same iteration and reports */
    CDV_MODE_SEPARABLE = 5      /* template given as per-axis factors (cdv_plan_set_psf_factors):
                                   both operators as one 1-D FP32 pass per axis; same iteration,
                                   decisions and reports as the direct modes */
} cdv_mode;

typedef struct cdv_plan cdv_plan;

/* Human-readable name of a status code (static string). */
const char* cdv_status_string(cdv_status s);

/* Details of the last error raised on the calling host thread ("" if none). */
const char* cdv_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int cdv_version(void);

/*
 * Plan for one problem size.  n in {1,2,3}; m[0..n-1] >= 1 samples of X per
 * axis; p[0..n-1] >= 0 half-widths of H (H has 2p_i+1 samples per axis).
 * Allocates the workspace on the current CUDA device (the plan is bound to
 * it).  *out receives the plan, or NULL on error.
 * Tensor-core modes pick between two kernels by a cycle model (the wide one,
 * 8 or 16 output columns per tile; the narrow one, 4 columns and 32 sliding
 * output-plane slots, for BF16 forms with q1 <= 31 and q3 = 1 mod 4).  The
 * environment variable CDV_TC_KERNEL, read here, overrides the choice:
 * "wide", "narrow", "narrow_rows" or "narrow_flat" (the narrow kernel with the
 * forward's tiles over rows only, or over column groups and rows), and
 * CDV_TC_DEAL = "free" or "chunks" restricts how the narrow kernel's tile
 * lists are cut (free cuts per M block, or chunk-major; default: the model's
 * choice per direction).  Both are measurement aids; the results do not
 * depend on them.
 */
cdv_status cdv_plan_create(cdv_plan** out, int n, const int64_t* m, const int32_t* p,
                           cdv_mode mode, void* stream);

/* Bytes of device memory the plan holds (workspace + templates). */
cdv_status cdv_plan_workspace_size(const cdv_plan* plan, size_t* bytes);

/*
 * Set the template H (device, float32, C-order, prod(2p_i+1) values).  The
 * plan copies it and derives, on `stream`, the flipped template
 * H~(j) = h(2p - j) of Property 2 and sum_j |h(j)|, from which the default
 * step length 1/L with L = (sum_j |h(j)|)^2 >= ||A||_2^2 is taken on the
 * device.  Asynchronous; H may be reused by the caller once `stream` has
 * reached this point.
 */
cdv_status cdv_plan_set_psf(cdv_plan* plan, const float* H, void* stream);

/*
 * Set a separable template H(j_1, .., j_n) = h_1(j_1) ... h_n(j_n) on a
 * CDV_MODE_SEPARABLE plan.  `h` is a host array of n device pointers; h[i]
 * holds the 2p_i + 1 float32 samples of the factor along axis i (axis n is
 * the contiguous one).  The plan copies the factors, builds the dense H from
 * them (for sum_j |h(j)| and the default step length, as cdv_plan_set_psf
 * does) and from then on computes both operators axis by axis: with a
 * product template the block-Toeplitz matrix of Property 1 is the Kronecker
 * product of the per-axis Toeplitz matrices, so the forward operator is a 1-D
 * full convolution along each axis (m_i -> m_i + 2p_i) and the adjoint of
 * Property 2 a 1-D valid correlation along each axis (m_i + 2p_i -> m_i).
 * Factors of 1..31 samples per axis.  CDV_ERR_UNSUPPORTED on a plan of any
 * other mode (and cdv_plan_set_psf returns it on a separable plan).
 * Asynchronous on `stream`, like cdv_plan_set_psf.
 */
cdv_status cdv_plan_set_psf_factors(cdv_plan* plan, const float* const* h, void* stream);

/* Lipschitz bound L = (sum |h|)^2 of the current template (host value).
 * Synchronises the device. */
cdv_status cdv_plan_lipschitz(const cdv_plan* plan, double* L);

/*
 * How the plan computes its two convolutions (index 0: forward, Property 1;
 * index 1: adjoint, Property 2).  The paper has no counterpart: this reports
 * the engine's tiling so that measured times can be set against the work
 * the hardware executes.  For the tensor-core modes `cols` is the number of
 * output columns per plane of one tile (8 or 16), `K` the Toeplitz window
 * along the contiguous axis and `executed_macs` the multiply-adds the tensor
 * pipe performs per launch, all products of split-BF16x3 included (padding
 * of K, of ragged tiles and of odd plane counts counted too).  For the FP32
 * engine cols = K = 0 and executed_macs = algorithmic_macs; for CDV_MODE_FFT all are 0; for
 * CDV_MODE_SEPARABLE executed_macs counts the three 1-D passes (outputs x taps of each) and
 * algorithmic_macs stays the dense count prod(m) prod(2p+1).  `grid` is the
 * number of CTAs of one launch.  Host-only: no device work.
 */
typedef struct cdv_plan_info {
    int32_t mode;
    int32_t cols[2];
    int32_t K[2];
    int32_t grid[2];
    int64_t tiles[2];
    double executed_macs[2];
    double algorithmic_macs;   /* prod(m) * prod(2p+1), the same for both directions */
} cdv_plan_info;

cdv_status cdv_plan_describe(const cdv_plan* plan, cdv_plan_info* out);

/* Free everything the plan owns.  NULL is accepted. */
cdv_status cdv_plan_destroy(cdv_plan* plan);

/*
 * Forward operator, Property 1 (Eq. 1): Y^v = A_n^h X^v, i.e.
 * y(s) = sum_k x(k) h(s - k) with zeros outside X.  X: m, Y: m + 2p.
 * `batch` volumes laid out back to back (X: batch*prod(m), Y: batch*prod(m+2p)).
 */
cdv_status cdv_forward(cdv_plan* plan, int batch, const float* X, float* Y, void* stream);

/*
 * Adjoint operator, Property 2 (Eq. 2): G^v = (A_n^h)^T R^v = {M_2p(R (*) H~)}^v,
 * i.e. g(k) = sum_{j in [0,2p]} h(j) r(k + j).  R: m + 2p, G: m, `batch` volumes.
 */
cdv_status cdv_adjoint(cdv_plan* plan, int batch, const float* R, float* G, void* stream);

/*
 * Gradient of a loss L(Y) with Y = X (*) H with respect to H:
 * dH(j) = sum_b sum_k X_b(k) dY_b(k + j)  (the adjoint sum of Property 2 with
 * the roles of x and h exchanged).  X: batch*prod(m), dY: batch*prod(m+2p),
 * dH: prod(2p+1), overwritten.  Uses the plan's workspace for block partials;
 * the final sum is FP64 in a fixed order (deterministic).
 */
cdv_status cdv_grad_psf(cdv_plan* plan, int batch, const float* X, const float* dY, float* dH,
                        void* stream);

/*
 * cdv_grad_psf for callers that cannot allocate device memory (for example
 * code running during a global-mode CUDA graph capture, or a plug-in whose
 * host framework owns all device memory).  The paper has no counterpart:
 * this is a deployment variant of the template gradient above.
 *
 * No plan: n, m[0..n-1] and p[0..n-1] describe the problem as in
 * cdv_plan_create; X, dY and dH are as in cdv_grad_psf and owned by the
 * caller.  The call allocates nothing.  Its FP64 partials live in a
 * library-wide static device array of 4 MiB (held by every GPU that loads
 * the library, until exit), so the template may have at most 524288 samples;
 * one block stages 16 + 2 p2 template rows of about 72 + 2 p3 floats and its
 * shared memory may not exceed 227 KB (roughly (16 + 2 p2) (72 + 2 p3) <=
 * 55,000 floats for narrow rows), and q2 * ceil(q3 / 4) may not exceed 1024.
 * Beyond any of these limits: CDV_ERR_UNSUPPORTED, nothing enqueued.  The first call on each
 * device looks up the array's address and must come before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race,
 * so order them on one stream.  Asynchronous on `stream`.
 */
cdv_status cdv_grad_psf_static(int n, const int64_t* m, const int32_t* p, int batch, const float* X,
                               const float* dY, float* dH, void* stream);

/* Initial solution of Step 1 (the paper leaves it open). */
typedef enum {
    CDV_X0_GIVEN = 0,   /* X holds x_0 on entry */
    CDV_X0_CROP = 1,    /* x_0 = max(Y[p : p + m], 0), the centre crop of Y */
    CDV_X0_ZERO = 2     /* x_0 = 0 */
} cdv_x0_policy;

typedef struct {
    int x0_policy;      /* cdv_x0_policy, default CDV_X0_GIVEN */
    double delta0;      /* step length tried first at every step; <= 0: 1/L (default) */
    double beta;        /* factor applied to delta after a rejected trial, default 0.5 */
    int max_halvings;   /* rejected trials allowed within one step, default 20 */
    int max_rejects;    /* rejected trials allowed in the whole run, default 16 */
    int use_graph;      /* 1: replay the captured K-step sequence as a CUDA graph (default) */
    int path;           /* cdv_iter_path, default CDV_PATH_AUTO */
    int bb;             /* 1: each step's first trial uses a Barzilai-Borwein length lagged by one
                           step, <s,s>/<s,v> with s = x_{k-1} - x_{k-2}, v = grad f(x_{k-1}) -
                           grad f(x_{k-2}) (k >= 2; delta0 before, and when <s,v> <= 0), clamped
                           to [delta0, 2^20 delta0]; 0 (default): delta0 at every step.  General
                           path only, like tikhonov and armijo */
    int reserved[2];
    double tikhonov;    /* lambda >= 0 of the term lambda/2 ||x||^2 added to f, default 0 (the
                           paper's objective); the introduction names Tikhonov regularisation */
    double armijo;      /* sigma in [0, 1): a trial is accepted when f(x_t) < f(x_k) +
                           sigma <grad f(x_k), x_t - x_k>; 0 (default) is the decrease
                           condition of Step 2.  Nonzero tikhonov or armijo (or bb): general path
                           only (CDV_ERR_UNSUPPORTED on the single-CTA path and the batched solver) */
} cdv_iter_opts;

/* Which kernels run the iteration. */
typedef enum {
    CDV_PATH_AUTO = 0,      /* the single-CTA path when the problem fits in one SM, else the general one */
    CDV_PATH_GENERAL = 1,   /* per-step forward/adjoint launches over the whole GPU (CUDA graph) */
    CDV_PATH_SMALL = 2,     /* one CTA holds the whole problem in shared memory and runs all K steps
                               in one launch; CDV_ERR_UNSUPPORTED if it does not fit (template width
                               along the contiguous axis <= 15, about 200 KB of state) */
    CDV_PATH_PERSISTENT = 3 /* batched solver only (its default, as CDV_PATH_AUTO): one persistent launch
                               runs every volume's whole run; cdv_iterate answers CDV_ERR_UNSUPPORTED */
} cdv_iter_path;

/* Fill `o` with the defaults above. */
void cdv_iter_opts_default(cdv_iter_opts* o);

typedef struct {
    int accepted;       /* steps accepted (K unless stopped early) */
    int rejected;       /* trials rejected by the decrease rule */
    int status;         /* cdv_status of the run: CDV_OK, CDV_ERR_NOT_DESCENDING
                           (converged: no decreasing step), CDV_ERR_NONFINITE */
    int trials;         /* forward convolutions run after the initial one */
    double f0;          /* f(x_0) = 1/2 ||A x_0 - y||^2 (+ lambda/2 ||x_0||^2) */
    double f_final;     /* f at the last accepted iterate */
    double gmac;        /* algorithmic multiply-adds executed, in units of 1e9 */
    double* f_hist;     /* optional host array of K+1: f(x_0), ..., f(x_accepted) */
    double* delta_hist; /* optional host array of K: accepted step lengths */
} cdv_iter_report;

/*
 * Projected gradient of Steps 1-3:
 *   x_{k+1} = max(x_k - delta_k A^T (A x_k - y), 0)
 * (the residual form of Eq. 6), for K accepted steps, with delta_k the first
 * of delta0, delta0*beta, delta0*beta^2, ... that makes f(x_{k+1}) < f(x_k).
 * With opts->tikhonov = lambda > 0 the objective is 1/2 ||A x - y||^2 +
 * lambda/2 ||x||^2 and the gradient gains lambda x_k (default delta0 =
 * 1/((sum |h|)^2 + lambda)); with opts->armijo = sigma > 0 the condition is
 * f(x_{k+1}) < f(x_k) + sigma <grad f(x_k), x_{k+1} - x_k>.
 * Every decision is taken on the device (FP64 objective), so the whole run is
 * one CUDA-graph replay with no host round trip.
 * Y: m + 2p (device), X: m (device; x_0 in per policy, x_K out).
 * If `rep` is not NULL the call synchronises `stream` and fills it.
 */
cdv_status cdv_iterate(cdv_plan* plan, const float* Y, float* X, int K, const cdv_iter_opts* opts,
                       cdv_iter_report* rep, void* stream);

/*
 * cdv_iterate with HOST arrays: copies Y_host (and X_host when the policy is
 * CDV_X0_GIVEN) to the plan's device buffers, iterates, copies x_K back to
 * X_host, and synchronises.  Pinned host memory gives the fastest copies.
 */
cdv_status cdv_iterate_host(cdv_plan* plan, const float* Y_host, float* X_host, int K,
                            const cdv_iter_opts* opts, cdv_iter_report* rep, void* stream);

/*
 * Richardson-Lucy, the comparison method of the Results section:
 *   x_{k+1} = x_k * A^T(y / A x_k) / A^T 1   (0 where A x_k = 0 or A^T 1 = 0).
 * X holds x_0 > 0 on entry and x_K on return.  Asynchronous.
 */
cdv_status cdv_richardson_lucy(cdv_plan* plan, const float* Y, float* X, int K, void* stream);

/*
 * Batched solver: `count` independent problems, volume i with n axes of
 * m[i*n + a] samples and template half-widths p[i*n + a], all iterated
 * together (Steps 1-3 per volume, each with its own step rule).  By default
 * (path CDV_PATH_AUTO or CDV_PATH_PERSISTENT) one persistent launch runs every
 * volume's whole run: its CTAs take the FP32-engine tiles of any volume whose
 * current phase (initial forward, adjoint trial, forward trial) has tiles left,
 * and the CTA that completes a phase runs that volume's FP64 step rule, so the
 * volumes advance independently.  With CDV_PATH_GENERAL the volumes advance
 * through common trial slots of batched launches whose work lists hold the
 * tiles of every volume (one launch per template width along the contiguous
 * axis).  Either run is replayed as one CUDA graph (use_graph = 1).  With autotune != 0 the tile shape
 * of each volume and direction is chosen by timing the candidates at plan
 * creation (results cached per process); iterates do not depend on the tile
 * shape and equal those of cdv_iterate on each volume alone.  CDV_MODE_FP32
 * only.  Allocates every workspace at creation; synchronises `stream`.
 */
typedef struct cdv_batch cdv_batch;
cdv_status cdv_batch_plan_create(cdv_batch** out, int count, int n, const int64_t* m, const int32_t* p,
                                 cdv_mode mode, int autotune, void* stream);

/* Bytes of device memory the batch plan holds. */
cdv_status cdv_batch_workspace_size(const cdv_batch* b, size_t* bytes);

/* Templates of every volume: H[i] is a device pointer to prod(2p_i+1) floats (copied). */
cdv_status cdv_batch_set_psfs(cdv_batch* b, const float* const* H, void* stream);

/*
 * K accepted steps for every volume (K <= 4096): Y[i] (device, m_i + 2p_i) and
 * X[i] (device, m_i; x_0 per policy in, x_K out).  `reports`, if not NULL,
 * points to `count` reports (their f_hist/delta_hist arrays optional) and the
 * call then synchronises `stream`.  The captured graph is reused while the
 * arrays, K and the options stay the same.  CDV_ERR_UNSUPPORTED for path
 * CDV_PATH_SMALL; with reports, CDV_ERR_TIMEOUT if a CTA of the persistent run
 * found no tile to take for the wait budget (about 0.5 s: a fault of the run,
 * not expected).
 */
cdv_status cdv_batch_iterate(cdv_batch* b, const float* const* Y, float* const* X, int K, const cdv_iter_opts* opts,
                             cdv_iter_report* reports, void* stream);

/*
 * Budget, in SM clock cycles, for which a CTA of the persistent batched run
 * may find no tile to take before it records CDV_ERR_TIMEOUT and leaves (the
 * other CTAs leave at their next look; cdv_batch_iterate with reports then
 * returns CDV_ERR_TIMEOUT).  0: the default, 1e9 cycles (about 0.5 s), far
 * longer than any tile or step rule takes.  The paper has no counterpart: this
 * bounds the persistent kernel's idle loop.  Takes effect at the next call (a
 * captured graph is re-captured).  Negative cycles: CDV_ERR_INVALID_ARG.
 */
cdv_status cdv_batch_set_wait_cycles(cdv_batch* b, long long cycles);

/* Free everything the batch plan owns.  NULL is accepted. */
cdv_status cdv_batch_destroy(cdv_batch* b);

/* Wait for `stream`, then return and clear the plan's device status word.
 * A report filled by cdv_iterate also returns that word (as its status) and
 * clears it. */
cdv_status cdv_plan_sync_status(cdv_plan* plan, void* stream);

/*
 * Budget, in SM clock cycles, of every barrier wait in the work loops of the
 * tensor-core kernels of this plan (0: the default, 1e9 cycles, about 0.5 s).
 * A wait that runs out records CDV_ERR_TIMEOUT in the device status word; the
 * block then stops issuing work, waits for its own copies and tensor-core
 * operations (with a fixed budget of 2e9 cycles), frees its tensor memory and
 * exits, and later launches of the plan skip their work until the word is
 * read and cleared (cdv_plan_sync_status or a cdv_iterate report).  The paper
 * has no counterpart: this bounds the kernels' spin waits.  Takes effect at
 * the next launch; a captured iteration graph is re-captured.  Negative
 * cycles: CDV_ERR_INVALID_ARG.  Other modes have no such waits and ignore it.
 */
cdv_status cdv_plan_set_wait_cycles(cdv_plan* plan, long long cycles);

/*
 * Measurement aid (the paper has no counterpart): `blocks` x `threads`
 * threads each run 8 independent FP32 fused multiply-add chains for `iters`
 * rounds, i.e. 16 * iters * blocks * threads flop, and write one float each
 * to out[0 .. blocks*threads) (device, caller-owned).  Timed by the caller,
 * this gives the GPU's FP32 FMA rate.  threads: a multiple of 32 up to 512;
 * other arguments out of range: CDV_ERR_INVALID_ARG.  Asynchronous on
 * `stream`.
 */
cdv_status cdv_probe_fp32_fma(float* out, int blocks, int threads, int iters, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CDV_H */

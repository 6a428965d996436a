/*
 * FP64 CPU oracle for direct-convolution deconvolution
 * ("Properties on n-dimensional convolution for image deconvolution").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing of the product path links or calls this
 * file; only the tests, the smoke check and the CPU-baseline leg of the bench
 * do.  It shares no code with the CUDA kernels.
 *
 * Plain nested loops in double precision, parallel over the slowest output
 * axis with OpenMP.  Every array is C-order with axis 1 slowest and axis 3
 * contiguous (the row partition of the vectorisation X^v in Property 1).
 * n < 3 is handled by the callers with leading axes of size 1 and p = 0.
 *
 * Index convention (0-based, m_i = number of samples):
 *   X  : m1 x m2 x m3                        (the target x(k))
 *   H  : q1 x q2 x q3,  q_i = 2 p_i + 1      (the template h(j))
 *   Y  : (m1+2p1) x (m2+2p2) x (m3+2p3)      (full convolution y(s))
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel regions (timing runs only; results do not depend on it). */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * Forward operator, Property 1: y(s) = sum_k x(k) h(s - k)  (Eq. 1, Y^v = A X^v).
 * Written as the shift-and-add of the block-Toeplitz rows of A: output plane
 * s1 receives the block A(j1) applied to x plane k1 = s1 - j1, and inside the
 * block every row k2 of x contributes h(j1, j2, .) * x(k1, k2, .) to output
 * row k2 + j2, shifted by j3 along the contiguous axis.  Each (k, j) pair with
 * s = k + j is visited exactly once.
 */
void orc_forward(int64_t m1, int64_t m2, int64_t m3, int p1, int p2, int p3,
                 const double* X, const double* H, double* Y)
{
    const int64_t q1 = 2 * p1 + 1, q2 = 2 * p2 + 1, q3 = 2 * p3 + 1;
    const int64_t n1 = m1 + 2 * p1, n2 = m2 + 2 * p2, n3 = m3 + 2 * p3;
    memset(Y, 0, sizeof(double) * (size_t)(n1 * n2 * n3));
    int64_t s1;
#pragma omp parallel for schedule(dynamic)
    for (s1 = 0; s1 < n1; s1++) {
        for (int64_t j1 = 0; j1 < q1; j1++) {
            const int64_t k1 = s1 - j1;
            if (k1 < 0 || k1 >= m1) continue;
            for (int64_t k2 = 0; k2 < m2; k2++) {
                const double* xr = X + (k1 * m2 + k2) * m3;
                for (int64_t j2 = 0; j2 < q2; j2++) {
                    double* yr = Y + (s1 * n2 + (k2 + j2)) * n3;
                    for (int64_t j3 = 0; j3 < q3; j3++) {
                        const double h = H[(j1 * q2 + j2) * q3 + j3];
                        for (int64_t k3 = 0; k3 < m3; k3++)
                            yr[k3 + j3] += h * xr[k3];
                    }
                }
            }
        }
    }
}

/*
 * Adjoint operator, Property 2 (Eq. 2): (A^T r)(k) = sum_{j in [0,2p]} h(j) r(k + j),
 * k in [0, m).  This is the crop M_{2p} of r (*) H~ with H~(j) = h(2p - j),
 * written as the sum it reduces to (checked against the literal crop in
 * orc_adjoint_crop).  R has the size of Y.
 */
void orc_adjoint(int64_t m1, int64_t m2, int64_t m3, int p1, int p2, int p3,
                 const double* R, const double* H, double* G)
{
    const int64_t q1 = 2 * p1 + 1, q2 = 2 * p2 + 1, q3 = 2 * p3 + 1;
    const int64_t n2 = m2 + 2 * p2, n3 = m3 + 2 * p3;
    memset(G, 0, sizeof(double) * (size_t)(m1 * m2 * m3));
    int64_t k1;
#pragma omp parallel for schedule(dynamic)
    for (k1 = 0; k1 < m1; k1++) {
        for (int64_t j1 = 0; j1 < q1; j1++) {
            for (int64_t k2 = 0; k2 < m2; k2++) {
                double* gr = G + (k1 * m2 + k2) * m3;
                for (int64_t j2 = 0; j2 < q2; j2++) {
                    const double* rr = R + ((k1 + j1) * n2 + (k2 + j2)) * n3;
                    for (int64_t j3 = 0; j3 < q3; j3++) {
                        const double h = H[(j1 * q2 + j2) * q3 + j3];
                        for (int64_t k3 = 0; k3 < m3; k3++)
                            gr[k3] += h * rr[k3 + j3];
                    }
                }
            }
        }
    }
}

/*
 * Property 2 taken literally: the full convolution of R (size m+2p) with the
 * flipped template H~(s) = h(2p - s), of size m + 4p per axis, then the crop
 * M_{2p} that keeps indices [2p, 2p + m) of every axis.
 */
void orc_adjoint_crop(int64_t m1, int64_t m2, int64_t m3, int p1, int p2, int p3,
                      const double* R, const double* H, double* G)
{
    const int64_t q1 = 2 * p1 + 1, q2 = 2 * p2 + 1, q3 = 2 * p3 + 1;
    const int64_t n1 = m1 + 2 * p1, n2 = m2 + 2 * p2, n3 = m3 + 2 * p3;
    const int64_t e1 = n1 + 2 * p1, e2 = n2 + 2 * p2, e3 = n3 + 2 * p3;
    double* Ht = (double*)malloc(sizeof(double) * (size_t)(q1 * q2 * q3));
    double* Yh = (double*)malloc(sizeof(double) * (size_t)(e1 * e2 * e3));
    for (int64_t a = 0; a < q1; a++)
        for (int64_t b = 0; b < q2; b++)
            for (int64_t c = 0; c < q3; c++)
                Ht[(a * q2 + b) * q3 + c] = H[((q1 - 1 - a) * q2 + (q2 - 1 - b)) * q3 + (q3 - 1 - c)];
    orc_forward(n1, n2, n3, p1, p2, p3, R, Ht, Yh);
    for (int64_t k1 = 0; k1 < m1; k1++)
        for (int64_t k2 = 0; k2 < m2; k2++)
            for (int64_t k3 = 0; k3 < m3; k3++)
                G[(k1 * m2 + k2) * m3 + k3] = Yh[((k1 + 2 * p1) * e2 + (k2 + 2 * p2)) * e3 + (k3 + 2 * p3)];
    free(Ht);
    free(Yh);
}

/* y(s) = sum_k x(k) h(s - k) at selected output points s (npts x 3 indices). */
void orc_forward_points(int64_t m1, int64_t m2, int64_t m3, int p1, int p2, int p3,
                        const double* X, const double* H,
                        int64_t npts, const int64_t* idx, double* out)
{
    const int64_t q1 = 2 * p1 + 1, q2 = 2 * p2 + 1, q3 = 2 * p3 + 1;
    int64_t i;
#pragma omp parallel for schedule(dynamic)
    for (i = 0; i < npts; i++) {
        const int64_t s1 = idx[3 * i], s2 = idx[3 * i + 1], s3 = idx[3 * i + 2];
        double acc = 0.0;
        for (int64_t j1 = 0; j1 < q1; j1++) {
            const int64_t k1 = s1 - j1;
            if (k1 < 0 || k1 >= m1) continue;
            for (int64_t j2 = 0; j2 < q2; j2++) {
                const int64_t k2 = s2 - j2;
                if (k2 < 0 || k2 >= m2) continue;
                for (int64_t j3 = 0; j3 < q3; j3++) {
                    const int64_t k3 = s3 - j3;
                    if (k3 < 0 || k3 >= m3) continue;
                    acc += X[(k1 * m2 + k2) * m3 + k3] * H[(j1 * q2 + j2) * q3 + j3];
                }
            }
        }
        out[i] = acc;
    }
}

/* (A^T r)(k) = sum_j h(j) r(k + j) at selected points k (npts x 3 indices). */
void orc_adjoint_points(int64_t m1, int64_t m2, int64_t m3, int p1, int p2, int p3,
                        const double* R, const double* H,
                        int64_t npts, const int64_t* idx, double* out)
{
    const int64_t q1 = 2 * p1 + 1, q2 = 2 * p2 + 1, q3 = 2 * p3 + 1;
    const int64_t n2 = m2 + 2 * p2, n3 = m3 + 2 * p3;
    (void)m1;
    int64_t i;
#pragma omp parallel for schedule(dynamic)
    for (i = 0; i < npts; i++) {
        const int64_t k1 = idx[3 * i], k2 = idx[3 * i + 1], k3 = idx[3 * i + 2];
        double acc = 0.0;
        for (int64_t j1 = 0; j1 < q1; j1++)
            for (int64_t j2 = 0; j2 < q2; j2++)
                for (int64_t j3 = 0; j3 < q3; j3++)
                    acc += H[(j1 * q2 + j2) * q3 + j3] * R[((k1 + j1) * n2 + (k2 + j2)) * n3 + (k3 + j3)];
        out[i] = acc;
    }
}

/*
 * Gradient of <Y, W> with Y = X (*) H with respect to the template:
 * dH(j) = sum_b sum_k X_b(k) dY_b(k + j).  This is Property 2's sum with the
 * roles of x and h exchanged (convolution commutes), so dH is the valid
 * correlation of dY with X.  X: batch x m, dY: batch x (m + 2p), dH: q.
 */
void orc_grad_psf(int64_t batch, int64_t m1, int64_t m2, int64_t m3, int p1, int p2, int p3,
                  const double* X, const double* dY, double* dH)
{
    const int64_t q1 = 2 * p1 + 1, q2 = 2 * p2 + 1, q3 = 2 * p3 + 1;
    const int64_t n1 = m1 + 2 * p1, n2 = m2 + 2 * p2, n3 = m3 + 2 * p3;
    const int64_t nx = m1 * m2 * m3, ny = n1 * n2 * n3;
    int64_t jj;
#pragma omp parallel for schedule(dynamic)
    for (jj = 0; jj < q1 * q2; jj++) {
        const int64_t j1 = jj / q2, j2 = jj % q2;
        for (int64_t j3 = 0; j3 < q3; j3++) {
            double acc = 0.0;
            for (int64_t b = 0; b < batch; b++)
                for (int64_t k1 = 0; k1 < m1; k1++)
                    for (int64_t k2 = 0; k2 < m2; k2++) {
                        const double* xr = X + b * nx + (k1 * m2 + k2) * m3;
                        const double* dr = dY + b * ny + ((k1 + j1) * n2 + (k2 + j2)) * n3 + j3;
                        for (int64_t k3 = 0; k3 < m3; k3++)
                            acc += xr[k3] * dr[k3];
                    }
            dH[(j1 * q2 + j2) * q3 + j3] = acc;
        }
    }
}

static double half_sq_norm(const double* v, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += v[i] * v[i];
    return 0.5 * s;
}

/*
 * Projected gradient for  min f(x) = 1/2 || A x - y ||^2 + lambda/2 || x ||^2  s.t. x >= 0
 * (Steps 1-3 of the 2-D application, any n; lambda = 0 is the paper's objective, lambda > 0 adds
 * the Tikhonov term the introduction names among the classic regularisers):
 *   x_{k+1} = max(x_k - delta_k * (A^T A x_k - A^T y + lambda x_k), 0),
 * with delta_k chosen so that f(x_{k+1}) < f(x_k) + sigma <grad f(x_k), x_{k+1} - x_k>.
 * sigma = 0 is the paper's decrease condition; sigma in (0, 1) is the Armijo sufficient-decrease
 * form of it.  The gradient is taken in the residual form A^T (A x - y), equal to Eq. 6 in exact
 * arithmetic.
 *
 * Step rule (the paper fixes only the decrease condition): every step's first
 * trial uses delta0 (bb = 0), or (bb = 1) a Barzilai-Borwein length lagged by
 * one step: delta_k = <s, s> / <s, v> with s = x_{k-1} - x_{k-2} and
 * v = grad f(x_{k-1}) - grad f(x_{k-2}) for k >= 2 (delta0 for k < 2, and when
 * <s, v> <= 0), clamped to [delta0, 2^20 delta0].  A trial that fails the
 * condition is rejected and delta is multiplied by beta, at most max_halvings
 * times.  A trial that leaves x unchanged, or an exhausted halving budget,
 * ends the run as converged.
 *
 * X holds x_0 on entry and the last accepted iterate on return.
 * f_hist[0..n_acc] receives f(x_0), f(x_1), ...; delta_hist[0..n_acc-1] the
 * accepted step lengths.  Returns 0 when K steps were accepted, 1 when the
 * run stopped early as converged.
 */
int orc_iterate(int64_t m1, int64_t m2, int64_t m3, int p1, int p2, int p3,
                const double* Y, const double* H, double* X, int K,
                double delta0, double beta, int max_halvings, double lambda, double sigma, int bb,
                double* f_hist, double* delta_hist, int* n_acc, int* n_rej)
{
    const int64_t n1 = m1 + 2 * p1, n2 = m2 + 2 * p2, n3 = m3 + 2 * p3;
    const int64_t nx = m1 * m2 * m3, ny = n1 * n2 * n3;
    double* r = (double*)malloc(sizeof(double) * (size_t)ny);
    double* rt = (double*)malloc(sizeof(double) * (size_t)ny);
    double* g = (double*)malloc(sizeof(double) * (size_t)nx);
    double* xt = (double*)malloc(sizeof(double) * (size_t)nx);
    double* xp = (double*)malloc(sizeof(double) * (size_t)nx);   /* x_{k-1} */
    double* gp = (double*)malloc(sizeof(double) * (size_t)nx);   /* grad f(x_{k-1}) */
    int status = 0, acc = 0, rej = 0;
    double bb_delta = delta0;                                     /* first trial of the next step */

    orc_forward(m1, m2, m3, p1, p2, p3, X, H, r);
    for (int64_t i = 0; i < ny; i++) r[i] -= Y[i];
    double f = half_sq_norm(r, ny) + lambda * half_sq_norm(X, nx);
    f_hist[0] = f;
    orc_adjoint(m1, m2, m3, p1, p2, p3, r, H, g);
    for (int64_t i = 0; i < nx; i++) g[i] += lambda * X[i];       /* grad f(x_k) */

    while (acc < K) {
        double delta = bb ? bb_delta : delta0;
        int halvings = 0, accepted = 0;
        double ft = 0.0;
        for (;;) {
            int moved = 0;
            double slope = 0.0;                                   /* <grad f(x_k), x_t - x_k> */
            for (int64_t i = 0; i < nx; i++) {
                const double v = X[i] - delta * g[i];
                xt[i] = v > 0.0 ? v : 0.0;
                if (xt[i] != X[i]) moved = 1;
                slope += g[i] * (xt[i] - X[i]);
            }
            if (!moved) break;
            orc_forward(m1, m2, m3, p1, p2, p3, xt, H, rt);
            for (int64_t i = 0; i < ny; i++) rt[i] -= Y[i];
            ft = half_sq_norm(rt, ny) + lambda * half_sq_norm(xt, nx);
            if (ft < f + sigma * slope) { accepted = 1; break; }
            rej++;
            if (++halvings > max_halvings) break;
            delta *= beta;
        }
        if (!accepted) { status = 1; break; }
        if (bb) {
            /* the length of the step after next: s = x_k - x_{k-1}, v = grad f(x_k) - grad f(x_{k-1}),
               formed when grad f(x_k) is, i.e. lagged by one step */
            if (acc >= 1) {
                double ss = 0.0, sv = 0.0;
                for (int64_t i = 0; i < nx; i++) {
                    const double si = X[i] - xp[i];
                    ss += si * si;
                    sv += si * (g[i] - gp[i]);
                }
                double d = sv > 0.0 ? ss / sv : delta0 * 1048576.0;
                if (d < delta0) d = delta0;
                if (d > delta0 * 1048576.0) d = delta0 * 1048576.0;
                bb_delta = d;
            }
            memcpy(xp, X, sizeof(double) * (size_t)nx);
            memcpy(gp, g, sizeof(double) * (size_t)nx);
        }
        memcpy(X, xt, sizeof(double) * (size_t)nx);
        double* tmp = r; r = rt; rt = tmp;
        f = ft;
        delta_hist[acc] = delta;
        acc++;
        f_hist[acc] = f;
        orc_adjoint(m1, m2, m3, p1, p2, p3, r, H, g);
        for (int64_t i = 0; i < nx; i++) g[i] += lambda * X[i];
    }
    *n_acc = acc;
    *n_rej = rej;
    free(r); free(rt); free(g); free(xt); free(xp); free(gp);
    return status;
}

/*
 * Richardson-Lucy, the comparison method of the Results section:
 *   x_{k+1} = x_k * A^T( y / (A x_k) ) / A^T 1,
 * with 0/0 taken as 0 where A x_k = 0.  X holds x_0 (> 0) on entry.
 */
void orc_richardson_lucy(int64_t m1, int64_t m2, int64_t m3, int p1, int p2, int p3,
                         const double* Y, const double* H, double* X, int K)
{
    const int64_t n1 = m1 + 2 * p1, n2 = m2 + 2 * p2, n3 = m3 + 2 * p3;
    const int64_t nx = m1 * m2 * m3, ny = n1 * n2 * n3;
    double* ax = (double*)malloc(sizeof(double) * (size_t)ny);
    double* ones = (double*)malloc(sizeof(double) * (size_t)ny);
    double* norm = (double*)malloc(sizeof(double) * (size_t)nx);
    double* corr = (double*)malloc(sizeof(double) * (size_t)nx);
    for (int64_t i = 0; i < ny; i++) ones[i] = 1.0;
    orc_adjoint(m1, m2, m3, p1, p2, p3, ones, H, norm);
    for (int it = 0; it < K; it++) {
        orc_forward(m1, m2, m3, p1, p2, p3, X, H, ax);
        for (int64_t i = 0; i < ny; i++) ax[i] = ax[i] != 0.0 ? Y[i] / ax[i] : 0.0;
        orc_adjoint(m1, m2, m3, p1, p2, p3, ax, H, corr);
        for (int64_t i = 0; i < nx; i++) X[i] = norm[i] != 0.0 ? X[i] * corr[i] / norm[i] : 0.0;
    }
    free(ax); free(ones); free(norm); free(corr);
}

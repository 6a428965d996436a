"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No GPU.  Each test checks the oracle against something other than itself:
the explicit matrix A_n^h built by the recursion of Property 1, library
routines (numpy/scipy convolution, correlation and NNLS), closed forms and
invariants.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.dense import dense_A

SHAPES = [
    ((7,), (3,)),
    ((5,), (9,)),            # template larger than the signal (q > m)
    ((1,), (5,)),
    ((6,), (1,)),            # p = 0
    ((4, 5), (3, 5)),
    ((3, 2), (5, 3)),
    ((3, 4, 5), (3, 1, 3)),
    ((2, 3, 4), (3, 5, 3)),
    ((4, 3, 2), (1, 3, 5)),
]


@pytest.mark.parametrize("m,q", SHAPES)
def test_forward_equals_dense_A_exactly(m, q):
    """Property 1 / Eq. 1: Y^v = A_n^h X^v, exact on integer data."""
    X, H = synth.integer_case(m, q, seed=len(m) * 100 + sum(m) + sum(q))
    A = dense_A(H, m)
    Y = oracle.forward(X, H)
    assert Y.shape == tuple(a + b - 1 for a, b in zip(m, q))
    np.testing.assert_array_equal(Y.ravel(), A @ X.astype(np.float64).ravel())


@pytest.mark.parametrize("m,q", SHAPES)
def test_adjoint_equals_dense_transpose_exactly(m, q):
    """Property 2 / Eq. 2: (A_n^h)^T R^v = {M_2p(R (*) H~)}^v, exact on integers."""
    X, H = synth.integer_case(m, q, seed=7 + sum(m))
    rng = np.random.default_rng(3)
    R = rng.integers(-4, 5, size=tuple(a + b - 1 for a, b in zip(m, q))).astype(np.float64)
    A = dense_A(H, m)
    G = oracle.adjoint(R, H)
    Gc = oracle.adjoint_crop(R, H)
    assert G.shape == tuple(m)
    np.testing.assert_array_equal(G.ravel(), A.T @ R.ravel())
    np.testing.assert_array_equal(Gc, G)


def test_extended_transpose_crop_offset():
    """Eq. S9/S11: the full conv with H~ has m + 4p samples and its crop starts at 2p."""
    m, q = (6,), (5,)
    X, H = synth.integer_case(m, q, seed=11)
    R = np.arange(1, 11, dtype=np.float64)
    Ht = H[::-1].astype(np.float64)
    full = np.convolve(R, Ht)          # textbook 1-D full convolution, m + 4p samples
    assert full.shape[0] == 6 + 8
    np.testing.assert_array_equal(oracle.adjoint(R, H), full[4:4 + 6])
    # shifting the crop by one is wrong: pins the offset
    assert not np.array_equal(oracle.adjoint(R, H), full[3:3 + 6])


@pytest.mark.parametrize("m,q", [((9, 8), (3, 5)), ((5, 6, 7), (3, 3, 5)), ((33,), (7,))])
def test_matches_scipy_convolve_and_correlate(m, q):
    """Library routines: scipy.signal.convolve(full) and correlate(valid)."""
    from scipy.signal import convolve, correlate
    X, H, R = synth.random_case(m, q, seed=5)
    np.testing.assert_allclose(oracle.forward(X, H),
                               convolve(X.astype(np.float64), H.astype(np.float64), mode="full", method="direct"),
                               rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.adjoint(R, H),
                               correlate(R.astype(np.float64), H.astype(np.float64), mode="valid", method="direct"),
                               rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("m,q", [((17, 12, 9), (5, 3, 7)), ((40, 31), (7, 9))])
def test_adjoint_identity(m, q):
    """<A x, r> = <x, A^T r> to FP64 rounding."""
    X, H, R = synth.random_case(m, q, seed=9)
    lhs = float(np.dot(oracle.forward(X, H).ravel(), R.astype(np.float64).ravel()))
    rhs = float(np.dot(X.astype(np.float64).ravel(), oracle.adjoint(R, H).ravel()))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_delta_templates_zero_boundary():
    """Zero boundary, no wrap-around: delta at 0 puts X in the corner, delta at the centre at offset p."""
    X, _ = synth.integer_case((5, 6, 4), (1, 1, 1), seed=1)
    q = (3, 5, 3)
    H0 = np.zeros(q); H0[0, 0, 0] = 1
    Y0 = oracle.forward(X, H0)
    exp0 = np.zeros(Y0.shape); exp0[:5, :6, :4] = X
    np.testing.assert_array_equal(Y0, exp0)
    Hc = np.zeros(q); Hc[1, 2, 1] = 1
    Yc = oracle.forward(X, Hc)
    expc = np.zeros(Yc.shape); expc[1:6, 2:8, 1:5] = X
    np.testing.assert_array_equal(Yc, expc)
    # adjoint of a centre delta is the centre crop
    np.testing.assert_array_equal(oracle.adjoint(Yc, Hc), X)


def test_convolution_not_correlation():
    """h(s - k): a ramp template is applied flipped relative to correlation."""
    X = np.zeros(5); X[2] = 1
    H = np.array([1.0, 2.0, 3.0])
    np.testing.assert_array_equal(oracle.forward(X, H), [0, 0, 1, 2, 3, 0, 0])
    R = np.array([0, 0, 1.0, 0, 0, 0, 0])
    np.testing.assert_array_equal(oracle.adjoint(R, H), [3, 2, 1, 0, 0])


def test_commutativity_and_mass():
    X, H = synth.integer_case((5, 7, 3), (3, 5, 9), seed=21)
    np.testing.assert_array_equal(oracle.forward(X, H), oracle.forward(H, X))
    Xr, Hr, _ = synth.random_case((11, 6, 9), (5, 3, 3), seed=2, positive=True)
    Y = oracle.forward(Xr, Hr)
    assert abs(Y.sum() - Xr.astype(np.float64).sum() * Hr.astype(np.float64).sum()) < 1e-11 * Y.sum()


def test_linearity_in_image_and_template():
    """Both operators are bilinear: linear in the image for a fixed template and in the template for a
    fixed image (Property 1 writes Y as A_n^h X with A_n^h built linearly from h)."""
    rng = np.random.default_rng(12)
    m, q = (6, 9, 11), (3, 5, 7)
    X1, X2 = rng.standard_normal(m), rng.standard_normal(m)
    H1, H2 = rng.standard_normal(q), rng.standard_normal(q)
    R1, R2 = (rng.standard_normal(tuple(a + b - 1 for a, b in zip(m, q))) for _ in range(2))
    a, b = 0.75, -1.5
    tol = dict(rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.forward(a * X1 + b * X2, H1),
                               a * oracle.forward(X1, H1) + b * oracle.forward(X2, H1), **tol)
    np.testing.assert_allclose(oracle.forward(X1, a * H1 + b * H2),
                               a * oracle.forward(X1, H1) + b * oracle.forward(X1, H2), **tol)
    np.testing.assert_allclose(oracle.adjoint(a * R1 + b * R2, H1),
                               a * oracle.adjoint(R1, H1) + b * oracle.adjoint(R2, H1), **tol)
    np.testing.assert_allclose(oracle.adjoint(R1, a * H1 + b * H2),
                               a * oracle.adjoint(R1, H1) + b * oracle.adjoint(R1, H2), **tol)


def test_separable_closed_form():
    """Separable X and H: Y is the outer product of 1-D textbook convolutions."""
    rng = np.random.default_rng(4)
    a, b, c = rng.random(9), rng.random(7), rng.random(12)
    H = synth.gaussian_psf((5, 7, 3), (1.2, 2.0, 0.9)).astype(np.float64)
    u, v, w = H.sum(axis=(1, 2)), H.sum(axis=(0, 2)), H.sum(axis=(0, 1))
    Hs = np.einsum("i,j,k->ijk", u, v, w)          # the Gaussian is separable: rebuild it as an outer product
    np.testing.assert_allclose(Hs, H, rtol=1e-5, atol=1e-9)
    X = np.einsum("i,j,k->ijk", a, b, c)
    Y = oracle.forward(X, Hs)
    Yc = np.einsum("i,j,k->ijk", np.convolve(a, u), np.convolve(b, v), np.convolve(c, w))
    np.testing.assert_allclose(Y, Yc, rtol=1e-12, atol=1e-14)


def test_product_template_matrix_is_kronecker_product():
    """For H = h1 x h2 x h3 the block-Toeplitz matrix of Property 1 is the Kronecker product of the 1-D
    full-convolution matrices (built here column by column with np.convolve on unit vectors); this is
    the identity the separable-template mode computes axis by axis.  Also checks the oracle's adjoint
    against the transposed Kronecker product."""
    rng = np.random.default_rng(11)
    m, q = (4, 5, 3), (3, 5, 3)
    hs = [rng.standard_normal(v) for v in q]

    def conv_matrix(h, n):
        return np.stack([np.convolve(np.eye(n)[i], h) for i in range(n)], axis=1)

    K = np.kron(np.kron(conv_matrix(hs[0], m[0]), conv_matrix(hs[1], m[1])), conv_matrix(hs[2], m[2]))
    H = np.einsum("i,j,k->ijk", *hs)
    np.testing.assert_allclose(dense_A(H, m), K, rtol=0, atol=1e-13)
    X = rng.standard_normal(m)
    R = rng.standard_normal(tuple(a + b - 1 for a, b in zip(m, q)))
    np.testing.assert_allclose(oracle.forward(X, H).ravel(), K @ X.ravel(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.adjoint(R, H).ravel(), K.T @ R.ravel(), rtol=1e-12, atol=1e-12)


def test_points_match_full():
    X, H, R = synth.random_case((13, 10, 17), (5, 7, 3), seed=8)
    Y = oracle.forward(X, H)
    G = oracle.adjoint(R, H)
    rng = np.random.default_rng(0)
    si = np.stack([rng.integers(0, n, 50) for n in Y.shape], axis=1)
    ki = np.stack([rng.integers(0, n, 50) for n in G.shape], axis=1)
    np.testing.assert_allclose(oracle.forward_points(X, H, si), Y[tuple(si.T)], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.adjoint_points(R, H, ki), G[tuple(ki.T)], rtol=1e-12, atol=1e-12)


def test_grad_psf_finite_differences():
    """dH of L = <X (*) H, W> against central differences in FP64 (h = 1e-3)."""
    rng = np.random.default_rng(12)
    B, m, q = 2, (5, 6, 4), (3, 3, 3)
    X = rng.random((B,) + m)
    H = rng.random(q)
    W = rng.standard_normal((B,) + tuple(a + b - 1 for a, b in zip(m, q)))
    dH = oracle.grad_psf(X, W, q)

    def L(Hv):
        return sum(float(np.sum(oracle.forward(X[b], Hv) * W[b])) for b in range(B))
    fd = np.zeros(q)
    for j in np.ndindex(q):
        e = np.zeros(q); e[j] = 1e-3
        fd[j] = (L(H + e) - L(H - e)) / 2e-3
    np.testing.assert_allclose(dH, fd, rtol=1e-8, atol=1e-8)
    # and against the library valid correlation of W with X
    from scipy.signal import correlate
    lib = sum(correlate(W[b], X[b], mode="valid", method="direct") for b in range(B))
    np.testing.assert_allclose(dH, lib, rtol=1e-12, atol=1e-12)


def test_grad_psf_dense_subcase():
    """8x8x8 / 3x3x3: dX = A^T dY from the explicit matrix, dH by the dense matrix of the roles swapped."""
    rng = np.random.default_rng(13)
    X = rng.random((8, 8, 8))
    H = rng.random((3, 3, 3))
    dY = rng.standard_normal((10, 10, 10))
    A = dense_A(H, (8, 8, 8))
    np.testing.assert_allclose(oracle.adjoint(dY, H).ravel(), A.T @ dY.ravel(), rtol=1e-12, atol=1e-12)
    # y is linear in h: y^v = B_X h^v with B_X[s, j] = x(s - j); dH = B_X^T dY^v
    Bx = np.zeros((1000, 27))
    for ji, j in enumerate(np.ndindex(3, 3, 3)):
        e = np.zeros((3, 3, 3)); e[j] = 1.0
        Bx[:, ji] = dense_A(e, (8, 8, 8)) @ X.ravel()
    np.testing.assert_allclose(oracle.grad_psf(X[None], dY[None], (3, 3, 3)).ravel(), Bx.T @ dY.ravel(),
                               rtol=1e-12, atol=1e-12)


def test_eq6_literal_equals_residual_form():
    P = synth.blobs2d()
    X0 = oracle.x0_crop(P.Y, P.p)
    lit, res = oracle.gradient_eq6(X0, P.H, P.Y)
    assert np.linalg.norm(lit - res) <= 1e-12 * np.linalg.norm(res)


def test_iterate_identity_template():
    """H = delta (A = I): one step with delta = 1 reaches max(Y, 0), then the run is stationary."""
    rng = np.random.default_rng(1)
    Y = rng.standard_normal((6, 7))
    H = np.ones((1, 1))
    out = oracle.iterate(Y, H, np.zeros((6, 7)) + 0.5, K=5)
    np.testing.assert_allclose(out["X"], np.maximum(Y, 0), rtol=0, atol=1e-15)
    assert out["accepted"] == 1 and out["status"] == 1


def test_iterate_monotone_and_nnls():
    """Steps 1-3 decrease f every accepted step and converge to the library NNLS solution."""
    from scipy.optimize import nnls
    rng = np.random.default_rng(2)
    H = synth.gaussian_psf((3, 3), (0.8, 0.8)).astype(np.float64)
    Xt = np.maximum(rng.standard_normal((8, 8)), 0)
    Y = oracle.forward(Xt, H) + 0.05 * rng.standard_normal((10, 10))
    A = dense_A(H, (8, 8))
    xs, _ = nnls(A, Y.ravel(), maxiter=5000)
    out = oracle.iterate(Y, H, np.zeros((8, 8)), K=20000)
    f = out["f"]
    assert np.all(np.diff(f) < 0)
    fs = 0.5 * np.sum((A @ xs - Y.ravel()) ** 2)
    assert f[-1] - fs <= 1e-9 * max(fs, 1.0)
    np.testing.assert_allclose(out["X"].ravel(), xs, atol=2e-3)
    # KKT of the NNLS problem at the limit
    g = A.T @ (A @ out["X"].ravel() - Y.ravel())
    assert np.all(out["X"] >= 0)
    assert np.all(g[out["X"].ravel() == 0] >= -1e-6)


def test_iterate_fejer_monotone_noise_free():
    """Noise-free Y from X_true > 0: ||x_k - X_true|| never grows with delta = 1/L."""
    rng = np.random.default_rng(3)
    H = synth.gaussian_psf((5, 3, 3), (1.0, 0.7, 0.7)).astype(np.float64)
    Xt = rng.random((6, 5, 7)) + 0.1
    Y = oracle.forward(Xt, H)
    x = np.zeros_like(Xt)
    d = [np.linalg.norm(x - Xt)]
    for _ in range(30):
        x = oracle.iterate(Y, H, x, K=1)["X"]
        d.append(np.linalg.norm(x - Xt))
    assert np.all(np.diff(d) <= 1e-12)
    assert d[-1] < d[0]


def test_iterate_backtracking():
    """A too-long delta0 is halved until f decreases; accepted deltas are delta0 * beta^i."""
    P = synth.blobs2d()
    X0 = oracle.x0_crop(P.Y, P.p)
    d0 = 8.0 / oracle.lipschitz(P.H)
    out = oracle.iterate(P.Y, P.H, X0, K=10, delta0=d0, beta=0.5)
    assert out["accepted"] == 10
    assert out["rejected"] > 0
    assert np.all(np.diff(out["f"]) < 0)
    ratio = np.log2(d0 / out["delta"])
    np.testing.assert_allclose(ratio, np.round(ratio), atol=1e-12)


def test_iterate_matches_step_by_step():
    """Two runs of K1 and K - K1 steps equal one run of K steps (state is x alone at fixed delta0)."""
    P = synth.blobs2d()
    X0 = oracle.x0_crop(P.Y, P.p)
    a = oracle.iterate(P.Y, P.H, X0, K=7)
    b1 = oracle.iterate(P.Y, P.H, X0, K=3)
    b2 = oracle.iterate(P.Y, P.H, b1["X"], K=4)
    np.testing.assert_array_equal(a["X"], b2["X"])
    np.testing.assert_array_equal(a["f"][3:], b2["f"])


def test_richardson_lucy_flux_and_fixed_point():
    """RL keeps sum(x) * sum(h) = sum(y), and y = A x_true is a fixed point at x_true."""
    rng = np.random.default_rng(5)
    H = synth.gaussian_psf((5, 5), (1.2, 1.2)).astype(np.float64)
    Xt = rng.random((9, 10)) + 0.2
    Y = oracle.forward(Xt, H)
    np.testing.assert_allclose(oracle.richardson_lucy(Y, H, Xt, 3), Xt, rtol=1e-12)
    Yn = Y + 0.01 * rng.random(Y.shape)
    x = oracle.richardson_lucy(Yn, H, np.ones_like(Xt), 4)
    assert abs(x.sum() * H.sum() - Yn.sum()) < 1e-10 * Yn.sum()


def test_lipschitz_bounds_operator_norm():
    H = synth.ring_psf(q=(7, 7, 5), sigma=(1, 1, 1.5), ring_r=2.5, ring_w=0.7, ring_sz=1.0)
    A = dense_A(H, (4, 5, 3))
    assert np.linalg.norm(A, 2) ** 2 <= oracle.lipschitz(H) * (1 + 1e-12)


def _delta_template():
    H = np.zeros((3, 3))
    H[1, 1] = 1.0                  # A embeds x in the centre of an (m+2) x (m+2) frame
    return H


def test_tikhonov_identity_template_closed_form():
    """H = delta, lambda > 0: f = 1/2||x - y_c||^2 + lambda/2 ||x||^2 + const, L = 1 + lambda, and one
    step of length 1/L from any x_0 lands on the minimiser y_c / (1 + lambda) (y_c > 0)."""
    rng = np.random.default_rng(11)
    lam = 0.37
    Y = rng.random((7, 9)) + 0.5
    X0 = rng.random((5, 7))
    out = oracle.iterate(Y, _delta_template(), X0, K=1, tikhonov=lam)
    yc = Y[1:-1, 1:-1]
    np.testing.assert_allclose(out["X"], yc / (1 + lam), rtol=1e-14)
    assert out["delta"][0] == pytest.approx(1 / (1 + lam), rel=1e-15)
    border = 0.5 * (np.sum(Y ** 2) - np.sum(yc ** 2))
    f1 = 0.5 * np.sum((yc / (1 + lam) - yc) ** 2) + border + 0.5 * lam * np.sum((yc / (1 + lam)) ** 2)
    assert out["f"][1] == pytest.approx(f1, rel=1e-13)
    f0 = 0.5 * np.sum((X0 - yc) ** 2) + border + 0.5 * lam * np.sum(X0 ** 2)
    assert out["f"][0] == pytest.approx(f0, rel=1e-13)


@pytest.mark.parametrize("sigma,delta,rejected", [(0.0, 1.0, 0), (0.4, 1.0, 0), (0.6, 0.5, 1)])
def test_armijo_identity_template_closed_form(sigma, delta, rejected):
    """H = delta, x_0 = 0, y_c > 0: the full step d = y_c gives f_t - f = -1/2 ||y_c||^2 against
    sigma <g, d> = -sigma ||y_c||^2, so it passes for sigma < 1/2; at sigma = 0.6 it is rejected and
    the half step (f_t - f = -3/8 ||y_c||^2 < -0.3 ||y_c||^2) is taken."""
    rng = np.random.default_rng(12)
    Y = rng.random((6, 8)) + 0.5
    out = oracle.iterate(Y, _delta_template(), np.zeros((4, 6)), K=1, armijo=sigma)
    assert out["accepted"] == 1 and out["rejected"] == rejected
    assert out["delta"][0] == delta
    np.testing.assert_allclose(out["X"], delta * Y[1:-1, 1:-1], rtol=1e-15)


def test_tikhonov_matches_nnls_augmented():
    """With lambda > 0 the problem is NNLS on the stacked system [A; sqrt(lambda) I] x ~ [y; 0]."""
    from scipy.optimize import nnls
    rng = np.random.default_rng(13)
    H = synth.gaussian_psf((3, 3), (0.8, 0.8)).astype(np.float64)
    Xt = np.maximum(rng.standard_normal((8, 8)), 0)
    Y = oracle.forward(Xt, H) + 0.05 * rng.standard_normal((10, 10))
    lam = 0.05
    A = dense_A(H, (8, 8))
    As = np.vstack([A, np.sqrt(lam) * np.eye(64)])
    xs, _ = nnls(As, np.concatenate([Y.ravel(), np.zeros(64)]), maxiter=5000)
    for sigma in (0.0, 1e-4, 0.3):
        out = oracle.iterate(Y, H, np.zeros((8, 8)), K=20000, tikhonov=lam, armijo=sigma)
        f = out["f"]
        assert np.all(np.diff(f) < 0)
        fs = 0.5 * np.sum((A @ xs - Y.ravel()) ** 2) + 0.5 * lam * np.sum(xs ** 2)
        assert f[-1] - fs <= 1e-10 * max(fs, 1.0)
        np.testing.assert_allclose(out["X"].ravel(), xs, atol=1e-6)


def test_bb_reduces_to_fixed_step_when_hessian_is_scalar():
    """A = c I (template c * delta): grad f(x) - grad f(x') = c^2 (x - x'), so every Barzilai-Borwein
    length equals 1/c^2 = 1/L and the run is the fixed-step run."""
    rng = np.random.default_rng(14)
    H = np.zeros((3, 3, 3))
    H[1, 1, 1] = 1.7
    Y = rng.standard_normal((6, 7, 8))
    X0 = rng.random((4, 5, 6))
    a = oracle.iterate(Y, H, X0, K=6)
    b = oracle.iterate(Y, H, X0, K=6, bb=True)
    np.testing.assert_allclose(b["delta"], a["delta"], rtol=1e-12)
    np.testing.assert_allclose(b["X"], a["X"], rtol=1e-12, atol=1e-14)


def test_bb_converges_to_nnls_in_fewer_steps():
    """The Barzilai-Borwein run reaches the NNLS optimum (same fixed point, monotone f) in far fewer
    accepted steps than the fixed step 1/L on an ill-conditioned blur."""
    from scipy.optimize import nnls
    rng = np.random.default_rng(15)
    H = synth.gaussian_psf((5, 5), (1.2, 1.2)).astype(np.float64)
    Xt = np.maximum(rng.standard_normal((10, 10)), 0)
    Y = oracle.forward(Xt, H) + 0.02 * rng.standard_normal((14, 14))
    A = dense_A(H, (10, 10))
    xs, _ = nnls(A, Y.ravel(), maxiter=10000)
    fs = 0.5 * np.sum((A @ xs - Y.ravel()) ** 2)

    def steps_to(out, tol):
        hit = np.nonzero(out["f"] - fs <= tol * fs)[0]
        return int(hit[0]) if hit.size else None

    plain = oracle.iterate(Y, H, np.zeros((10, 10)), K=4000)
    bb = oracle.iterate(Y, H, np.zeros((10, 10)), K=4000, bb=True)
    assert np.all(np.diff(bb["f"]) < 0)
    nb, npl = steps_to(bb, 1e-6), steps_to(plain, 1e-6)
    assert nb is not None and (npl is None or nb * 3 < npl)
    assert np.max(bb["delta"]) > oracle.lipschitz(H) ** -1 * 2       # longer steps than 1/L are taken
    np.testing.assert_allclose(bb["X"].ravel(), xs, atol=1e-4)


def test_bb_lag_is_one_step_cauchy_length_two_steps_back():
    """On a quadratic whose iterates stay positive (no projection), s = x_{k-1} - x_{k-2} equals
    -delta_{k-2} grad f(x_{k-2}) and v = A^T A s, so the lagged Barzilai-Borwein length <s,s>/<s,v> of
    step k is the exact line-search (Cauchy) length of the gradient two steps back,
    |g|^2 / (g^T A^T A g) with g = grad f(x_{k-2}); an unlagged length would be that of grad f(x_{k-1}).
    The Hessian here is not a multiple of the identity, so the two differ."""
    rng = np.random.default_rng(16)
    h = np.array([1.0, 0.1, 0.05])                   # A^T A well conditioned (kappa < 2): no rejections
    m = 6
    A = np.stack([np.convolve(np.eye(m)[i], h) for i in range(m)], axis=1)   # columns: library convolution
    Q = A.T @ A
    xt = 5.0 + rng.random(m)
    y = A @ xt
    x0 = xt + rng.uniform(-1.0, 1.0, m)
    K = 8
    out = oracle.iterate(y, h, x0, K=K, bb=True)
    assert out["accepted"] == K and out["rejected"] == 0
    d0 = 1.0 / np.sum(np.abs(h)) ** 2
    grad = lambda x: A.T @ (A @ x - y)
    xs = [x0]
    for k in range(K):                               # replay with the oracle's step lengths
        xs.append(np.maximum(xs[-1] - out["delta"][k] * grad(xs[-1]), 0.0))
    assert min(x.min() for x in xs) > 0.0            # the projection never acts
    np.testing.assert_allclose(xs[-1], out["X"], rtol=1e-12)
    cauchy = lambda g: float(g @ g / (g @ Q @ g))
    clamp = lambda d: min(max(d, d0), d0 * 2.0 ** 20)
    np.testing.assert_allclose(out["delta"][:2], d0, rtol=1e-15)
    lag1 = [clamp(cauchy(grad(xs[k - 2]))) for k in range(2, K)]
    lag0 = [clamp(cauchy(grad(xs[k - 1]))) for k in range(2, K)]
    np.testing.assert_allclose(out["delta"][2:], lag1, rtol=1e-9)
    assert np.max(np.abs(np.array(lag0) / np.array(lag1) - 1.0)) > 1e-3

"""GPU parity of the operators (through the C ABI) against the FP64 oracle.

Sizes span several CTA tiles along every axis with ragged tails; the
full-size 512x512x128 / 31x31x21 operators are checked on sampled outputs in
the same launch configuration the benchmark times.
"""
import numpy as np
import pytest

import oracle
import synth
from _util import TOL_CONV, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _plan(m, q):
    from paper_1711_11224_gb300 import Plan
    return Plan(m, [(v - 1) // 2 for v in q])


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


SHAPES = [
    ((9, 37, 45), (5, 7, 9)),         # several row tiles, ragged columns
    ((13, 20, 150), (3, 5, 21)),      # output rows wider than one CTA tile (two column tiles)
    ((6, 4, 300), (1, 3, 31)),        # widest template along the contiguous axis, q1 = 1
    ((3, 4, 5), (7, 9, 11)),          # template larger than the volume (q > m)
    ((17, 11, 8), (9, 3, 1)),         # q3 = 1
    ((70, 90), (7, 7)),               # n = 2
    ((1000,), (31,)),                 # n = 1
    ((5, 330, 7), (3, 11, 5)),        # many rows, narrow rows
]


@pytest.mark.parametrize("m,q", SHAPES)
def test_forward_adjoint_random(m, q):
    X, H, R = synth.random_case(m, q, seed=sum(m) + sum(q))
    with _plan(m, q) as pl:
        pl.set_psf(_dev(H))
        Y = pl.forward(_dev(X)).cpu().numpy()
        G = pl.adjoint(_dev(R)).cpu().numpy()
    assert rel_l2(Y, oracle.forward(X, H)) <= TOL_CONV
    assert rel_l2(G, oracle.adjoint(R, H)) <= TOL_CONV


@pytest.mark.parametrize("m,q", [((8, 21, 45), (5, 7, 9)), ((4, 5), (3, 5)), ((3, 4, 5), (7, 9, 11))])
def test_integer_data_bit_exact(m, q):
    """Integer data: every partial sum is an integer below 2^24, so FP32 is exact."""
    X, H = synth.integer_case(m, q, seed=3)
    rng = np.random.default_rng(0)
    R = rng.integers(-4, 5, size=tuple(a + b - 1 for a, b in zip(m, q))).astype(np.float32)
    with _plan(m, q) as pl:
        pl.set_psf(_dev(H))
        Y = pl.forward(_dev(X)).cpu().numpy()
        G = pl.adjoint(_dev(R)).cpu().numpy()
    np.testing.assert_array_equal(Y.astype(np.float64), oracle.forward(X, H))
    np.testing.assert_array_equal(G.astype(np.float64), oracle.adjoint(R, H))


def test_delta_template_places_x():
    m, q = (10, 12, 30), (5, 3, 7)
    X, _, _ = synth.random_case(m, q, seed=4)
    H = np.zeros(q, np.float32)
    H[2, 1, 3] = 1.0
    with _plan(m, q) as pl:
        pl.set_psf(_dev(H))
        Y = pl.forward(_dev(X)).cpu().numpy()
        G = pl.adjoint(_dev(Y)).cpu().numpy()
    E = np.zeros(Y.shape, np.float32)
    E[2:12, 1:13, 3:33] = X
    np.testing.assert_array_equal(Y, E)
    np.testing.assert_array_equal(G, X)


def test_batched_forward_adjoint():
    m, q, B = (7, 19, 33), (3, 5, 7), 3
    rng = np.random.default_rng(5)
    X = rng.random((B,) + m).astype(np.float32)
    H = rng.random(q).astype(np.float32)
    R = rng.standard_normal((B,) + tuple(a + b - 1 for a, b in zip(m, q))).astype(np.float32)
    with _plan(m, q) as pl:
        pl.set_psf(_dev(H))
        Y = pl.forward(_dev(X)).cpu().numpy()
        G = pl.adjoint(_dev(R)).cpu().numpy()
    for b in range(B):
        assert rel_l2(Y[b], oracle.forward(X[b], H)) <= TOL_CONV
        assert rel_l2(G[b], oracle.adjoint(R[b], H)) <= TOL_CONV


def test_adjoint_identity_gpu():
    m, q = (11, 23, 40), (5, 5, 9)
    X, H, R = synth.random_case(m, q, seed=6)
    with _plan(m, q) as pl:
        pl.set_psf(_dev(H))
        Y = pl.forward(_dev(X)).cpu().numpy().astype(np.float64)
        G = pl.adjoint(_dev(R)).cpu().numpy().astype(np.float64)
    lhs = float(np.dot(Y.ravel(), R.astype(np.float64).ravel()))
    rhs = float(np.dot(X.astype(np.float64).ravel(), G.ravel()))
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + 1e-30) * 10


def test_grad_psf_matches_oracle():
    B, m, q = 3, (9, 20, 70), (5, 7, 9)
    rng = np.random.default_rng(7)
    X = rng.random((B,) + m).astype(np.float32)
    dY = rng.standard_normal((B,) + tuple(a + b - 1 for a, b in zip(m, q))).astype(np.float32)
    with _plan(m, q) as pl:
        pl.set_psf(_dev(np.ones(q, np.float32)))
        dH = pl.grad_psf(_dev(X), _dev(dY)).cpu().numpy()
    assert rel_l2(dH, oracle.grad_psf(X, dY, q)) <= TOL_CONV


def test_autograd_dense_subcase():
    """8x8x8 / 3x3x3: dX against the explicit A^T, dH against the oracle (pinned by finite differences)."""
    from oracle.dense import dense_A
    from paper_1711_11224_gb300 import conv
    rng = np.random.default_rng(8)
    X = rng.random((2, 8, 8, 8)).astype(np.float32)
    H = rng.random((3, 3, 3)).astype(np.float32)
    W = rng.standard_normal((2, 10, 10, 10)).astype(np.float32)
    Xt = _dev(X).requires_grad_(True)
    Ht = _dev(H).requires_grad_(True)
    Y = conv(Xt, Ht)
    (Y * _dev(W)).sum().backward()
    A = dense_A(H, (8, 8, 8))
    for b in range(2):
        assert rel_l2(Y[b].detach().cpu().numpy().ravel(), A @ X[b].astype(np.float64).ravel()) <= TOL_CONV
        assert rel_l2(Xt.grad[b].cpu().numpy().ravel(), A.T @ W[b].astype(np.float64).ravel()) <= TOL_CONV
    assert rel_l2(Ht.grad.cpu().numpy(), oracle.grad_psf(X, W, (3, 3, 3))) <= TOL_CONV


def test_autograd_learnable_sigma():
    """c3: B=4 volumes 128x128x64, Gaussian 11x11x9 with learnable sigma; d/dsigma via torch, dH via the kernel."""
    from paper_1711_11224_gb300 import conv
    Xs, H0, sigma = synth.grad3d()
    X = _dev(Xs)
    sig = torch.tensor(sigma, dtype=torch.float64, device="cuda", requires_grad=True)

    def psf(s):
        q = (11, 11, 9)
        g = [torch.arange(n, dtype=torch.float64, device="cuda") - (n - 1) / 2 for n in q]
        e = (g[0][:, None, None] ** 2) / (2 * s[0] ** 2) + (g[1][None, :, None] ** 2) / (2 * s[1] ** 2) + \
            (g[2][None, None, :] ** 2) / (2 * s[2] ** 2)
        h = torch.exp(-e)
        return h / h.sum()

    Ht = psf(sig).float()
    Ht.retain_grad()
    Y = conv(X, Ht)
    rng = np.random.default_rng(9)
    W = rng.standard_normal(tuple(Y.shape)).astype(np.float32)
    loss = (Y * _dev(W)).sum()
    loss.backward()
    dH_ref = oracle.grad_psf(Xs, W, (11, 11, 9))
    assert rel_l2(Ht.grad.cpu().numpy(), dH_ref) <= TOL_CONV
    # chain rule through sigma: the same contraction with the FP64 oracle's dH
    dsig = sig.grad.cpu().numpy()
    s2 = sig.detach().clone().requires_grad_(True)
    (psf(s2) * torch.from_numpy(dH_ref).cuda()).sum().backward()
    np.testing.assert_allclose(dsig, s2.grad.cpu().numpy(), rtol=1e-4, atol=1e-6)


def _sample_idx(shape, n, seed):
    rng = np.random.default_rng(seed)
    idx = np.stack([rng.integers(0, s, n) for s in shape], axis=1)
    # include the corners and faces, where the zero boundary matters
    corners = np.array(np.meshgrid(*[[0, s - 1] for s in shape], indexing="ij")).reshape(len(shape), -1).T
    return np.concatenate([idx, corners])


@pytest.mark.parametrize("seed", [0])
def test_full_size_ring3d_sampled(seed):
    """512x512x128 with the 31x31x21 ring template, bench launch configuration, sampled outputs."""
    P = synth.ring3d()
    rng = np.random.default_rng(seed)
    R = rng.standard_normal(P.Y.shape).astype(np.float32)
    with _plan(P.m, P.H.shape) as pl:
        pl.set_psf(_dev(P.H))
        Y = pl.forward(_dev(P.X_true)).cpu().numpy()
        G = pl.adjoint(_dev(R)).cpu().numpy()
    si = _sample_idx(Y.shape, 1500, 1)
    ki = _sample_idx(G.shape, 1500, 2)
    yo = oracle.forward_points(P.X_true, P.H, si)
    go = oracle.adjoint_points(R, P.H, ki)
    assert rel_l2(Y[tuple(si.T)], yo) <= TOL_CONV
    assert rel_l2(G[tuple(ki.T)], go) <= TOL_CONV
    # mass invariant on the whole output (sum Y = sum X * sum H)
    tot = float(P.X_true.astype(np.float64).sum() * P.H.astype(np.float64).sum())
    assert abs(Y.astype(np.float64).sum() - tot) <= 1e-5 * tot


def test_errors_are_loud():
    from paper_1711_11224_gb300 import CdvError, Plan
    with pytest.raises(CdvError):
        Plan((4, 4, 4), (1, 1, 40))              # unsupported width along the contiguous axis
    with Plan((4, 4), (1, 1)) as pl:
        with pytest.raises(CdvError):
            pl.forward(_dev(np.zeros((4, 4))))   # no template yet

"""The separable-template mode (CDV_MODE_SEPARABLE) against the FP64 oracle.

The template is given as per-axis factors h_i; the oracle receives the dense outer product
H = h_1 x h_2 x h_3 (built here in FP64 from the same FP32 factors) and computes the sums of
Properties 1 and 2 directly, so every check compares the axis-by-axis passes with the dense
definition.
"""
import numpy as np
import pytest

import oracle
import synth
from _util import TOL_CONV, TOL_ITER, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _dense(hs):
    H = np.asarray(hs[0], dtype=np.float64)
    for h in hs[1:]:
        H = np.multiply.outer(H, np.asarray(h, dtype=np.float64))
    return H


def _plan(m, q):
    from paper_1711_11224_gb300 import Plan
    return Plan(m, [(v - 1) // 2 for v in q], mode="separable")


SHAPES = [
    ((9, 37, 45), (5, 7, 9)),          # several strips and row segments
    ((13, 20, 150), (3, 5, 21)),
    ((6, 4, 300), (1, 3, 31)),         # widest factor, q1 = 1
    ((3, 4, 5), (7, 9, 11)),           # factors longer than the volume (q > m)
    ((17, 11, 8), (9, 3, 1)),          # q3 = 1
    ((40, 33, 1), (31, 5, 1)),         # one sample along the contiguous axis: strided passes of inner 1
    ((70, 90), (7, 7)),                # n = 2
    ((2000,), (31,)),                  # n = 1, rows longer than one segment
]


@pytest.mark.parametrize("m,q", SHAPES)
def test_separable_forward_adjoint(m, q):
    rng = np.random.default_rng(sum(m) + sum(q))
    hs = [rng.standard_normal(v).astype(np.float32) for v in q]
    X = rng.standard_normal(m).astype(np.float32)
    R = rng.standard_normal(tuple(a + b - 1 for a, b in zip(m, q))).astype(np.float32)
    H = _dense(hs)
    with _plan(m, q) as pl:
        pl.set_psf_factors([_dev(h) for h in hs])
        Y = pl.forward(_dev(X)).cpu().numpy()
        G = pl.adjoint(_dev(R)).cpu().numpy()
        Yb = pl.forward(_dev(np.stack([X, 2 * X]))).cpu().numpy()        # batched plain call
        pl.sync()
        info = pl.describe()
    assert rel_l2(Y, oracle.forward(X, H)) <= TOL_CONV
    assert rel_l2(G, oracle.adjoint(R, H)) <= TOL_CONV
    np.testing.assert_array_equal(Yb[0], Y)
    assert rel_l2(Yb[1], 2 * oracle.forward(X, H)) <= TOL_CONV
    mq = [(a, b) for a, b in zip((1,) * (3 - len(m)) + tuple(m), (1,) * (3 - len(q)) + tuple(q))]
    (m1, q1), (m2, q2), (m3, q3) = mq
    b1, b2, b3 = m1 + q1 - 1, m2 + q2 - 1, m3 + q3 - 1
    assert info["executed_macs"][0] == m1 * m2 * b3 * q3 + m1 * b2 * b3 * q2 + b1 * b2 * b3 * q1
    assert info["algorithmic_macs"] == float(np.prod(m)) * float(np.prod(q))


def test_separable_integer_factors_exact():
    """Small integer factors and data: every partial sum is an integer below 2^24, so FP32 is exact."""
    rng = np.random.default_rng(3)
    m, q = (8, 21, 45), (5, 7, 9)
    hs = [rng.integers(-2, 3, v).astype(np.float32) for v in q]
    X = rng.integers(-3, 4, m).astype(np.float32)
    R = rng.integers(-3, 4, tuple(a + b - 1 for a, b in zip(m, q))).astype(np.float32)
    with _plan(m, q) as pl:
        pl.set_psf_factors([_dev(h) for h in hs])
        Y = pl.forward(_dev(X)).cpu().numpy()
        G = pl.adjoint(_dev(R)).cpu().numpy()
    np.testing.assert_array_equal(Y.astype(np.float64), oracle.forward(X, _dense(hs)))
    np.testing.assert_array_equal(G.astype(np.float64), oracle.adjoint(R, _dense(hs)))


def test_separable_iterate_100_matches_oracle_and_graph_equals_stream():
    """100 iterations on a filament volume with a Gaussian template given by its factors."""
    from paper_1711_11224_gb300 import Plan
    q, sigma = (5, 5, 7), (1.2, 1.2, 2.0)
    hs = synth.gaussian_factors(q, sigma)
    H = _dense(hs)
    rng = np.random.default_rng(0)
    X_true = synth.filaments((14, 40, 36), 6, rng)
    Y = rng.poisson(np.maximum(oracle.forward(X_true, H), 0)).astype(np.float32)
    p = [(v - 1) // 2 for v in q]
    ref = oracle.iterate(Y, H, oracle.x0_crop(Y, p), 100)
    outs = []
    for g in (True, False):
        with Plan(X_true.shape, p, mode="separable") as pl:
            pl.set_psf_factors([_dev(h) for h in hs])
            X, rep = pl.iterate(_dev(Y), K=100, x0="crop", use_graph=g)
            outs.append(X.cpu().numpy())
        assert rep["accepted"] == ref["accepted"] == 100 and rep["status"] == "CDV_OK"
        np.testing.assert_allclose(rep["f"], ref["f"], rtol=1e-5)
        assert rel_l2(outs[-1], ref["X"]) <= TOL_ITER
    np.testing.assert_array_equal(outs[0], outs[1])


def test_separable_iterate_with_variants():
    from paper_1711_11224_gb300 import Plan
    q = (5, 5, 7)
    hs = synth.gaussian_factors(q, (1.0, 1.4, 2.0))
    H = _dense(hs)
    P = synth.scaled_fil3d((12, 60, 50), q, K=12)
    Y = P.Y
    kw = {"tikhonov": 0.05, "armijo": 1e-4, "bb": True}
    ref = oracle.iterate(Y, H, oracle.x0_crop(Y, P.p), 12, **kw)
    with Plan(P.m, P.p, mode="separable") as pl:
        pl.set_psf_factors([_dev(h) for h in hs])
        X, rep = pl.iterate(_dev(Y), K=12, x0="crop", max_rejects=200, **kw)
    assert rep["accepted"] == ref["accepted"] == 12 and rep["rejected"] == ref["rejected"]
    np.testing.assert_allclose(rep["delta"], ref["delta"], rtol=2e-3)
    assert rel_l2(X.cpu().numpy(), ref["X"]) <= TOL_ITER


def test_separable_backtracking_matches_oracle():
    """A step length far above 1/L forces rejected trials (update-only adjoint passes)."""
    from paper_1711_11224_gb300 import Plan
    q = (3, 5, 5)
    hs = synth.gaussian_factors(q, (0.8, 1.2, 1.2))
    H = _dense(hs)
    P = synth.scaled_fil3d((10, 30, 40), q, K=10)
    L = oracle.lipschitz(H)
    ref = oracle.iterate(P.Y, H, oracle.x0_crop(P.Y, P.p), 10, delta0=64.0 / L)
    with Plan(P.m, P.p, mode="separable") as pl:
        pl.set_psf_factors([_dev(h) for h in hs])
        X, rep = pl.iterate(_dev(P.Y), K=10, x0="crop", delta0=64.0 / L, max_rejects=200)
    assert ref["rejected"] > 0
    assert rep["accepted"] == ref["accepted"] and rep["rejected"] == ref["rejected"]
    np.testing.assert_allclose(rep["delta"], ref["delta"], rtol=1e-12)
    assert rel_l2(X.cpu().numpy(), ref["X"]) <= TOL_ITER


def test_separable_full_size_fil3d_sampled():
    """256x256x64 with the 15x15x11 Gaussian of the filament workload, sampled outputs."""
    P = synth.fil3d()
    hs = synth.gaussian_factors((15, 15, 11), (1.5, 1.5, 3.0))
    H = _dense(hs)
    rng = np.random.default_rng(0)
    R = rng.standard_normal(P.Y.shape).astype(np.float32)
    with _plan(P.m, (15, 15, 11)) as pl:
        pl.set_psf_factors([_dev(h) for h in hs])
        Y = pl.forward(_dev(P.X_true)).cpu().numpy()
        G = pl.adjoint(_dev(R)).cpu().numpy()
    si = np.stack([rng.integers(0, s, 1500) for s in Y.shape], axis=1)
    ki = np.stack([rng.integers(0, s, 1500) for s in G.shape], axis=1)
    assert rel_l2(Y[tuple(si.T)], oracle.forward_points(P.X_true, H, si)) <= TOL_CONV
    assert rel_l2(G[tuple(ki.T)], oracle.adjoint_points(R, H, ki)) <= TOL_CONV
    # the factors of the filament workload's template reproduce it
    np.testing.assert_allclose(H, P.H, rtol=1e-5, atol=1e-9)


def test_separable_errors():
    from paper_1711_11224_gb300 import CdvError, Plan
    with _plan((8, 8, 8), (3, 3, 3)) as pl:
        with pytest.raises(CdvError):
            pl.set_psf(_dev(np.ones((3, 3, 3))))                  # a separable plan takes factors
        with pytest.raises(CdvError):
            pl.forward(_dev(np.zeros((8, 8, 8))))                 # no template yet
    with Plan((8, 8, 8), (1, 1, 1)) as pl:
        with pytest.raises(CdvError):
            pl.set_psf_factors([_dev(np.ones(3))] * 3)            # factors need a separable plan
    with pytest.raises(CdvError):
        Plan((8, 8, 40), (1, 1, 16), mode="separable")            # 33 samples along an axis

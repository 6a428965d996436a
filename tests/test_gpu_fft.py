"""The FFT comparator (CDV_MODE_FFT, cuFFT) against the FP64 oracle: the same operators and the same
iteration computed through zero-padded transforms instead of direct sums."""
import numpy as np
import pytest

import oracle
import synth
from _util import TOL_ITER, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP32 transforms of N samples carry errors of order eps * log2(N) relative to the norm of the result
TOL_FFT = 1e-5


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("m,q", [((3, 130, 40), (3, 5, 7)), ((50, 70), (7, 7)), ((3, 4, 5), (7, 9, 11)),
                                 ((20, 60, 33), (9, 3, 41)), ((257,), (31,))])
def test_fft_forward_adjoint(m, q):
    from paper_1711_11224_gb300 import Plan
    X, H, R = synth.random_case(m, q, seed=5)
    with Plan(m, [(v - 1) // 2 for v in q], mode="fft") as pl:
        pl.set_psf(_dev(H))
        Y = pl.forward(_dev(X)).cpu().numpy()
        G = pl.adjoint(_dev(R)).cpu().numpy()
        pl.sync()
    assert rel_l2(Y, oracle.forward(X, H)) <= TOL_FFT
    assert rel_l2(G, oracle.adjoint(R, H)) <= TOL_FFT


def test_fft_iterate_matches_oracle_and_graph_equals_stream():
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((16, 60, 50), (5, 5, 7), K=15)
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 15)
    outs = []
    for g in (True, False):
        with Plan(P.m, P.p, mode="fft") as pl:
            pl.set_psf(_dev(P.H))
            X, rep = pl.iterate(_dev(P.Y), K=15, x0="crop", use_graph=g)
            outs.append(X.cpu().numpy())
        assert rep["accepted"] == 15 and rep["status"] == "CDV_OK"
        np.testing.assert_allclose(rep["f"], ref["f"], rtol=1e-5)
        assert rel_l2(outs[-1], ref["X"]) <= TOL_ITER
    np.testing.assert_array_equal(outs[0], outs[1])


def test_fft_iterate_with_variants():
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((12, 60, 50), (5, 5, 7), K=12)
    kw = {"tikhonov": 0.05, "armijo": 1e-4, "bb": True}
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 12, **kw)
    with Plan(P.m, P.p, mode="fft") as pl:
        pl.set_psf(_dev(P.H))
        X, rep = pl.iterate(_dev(P.Y), K=12, x0="crop", max_rejects=200, **kw)
    assert rep["accepted"] == ref["accepted"] == 12 and rep["rejected"] == ref["rejected"]
    np.testing.assert_allclose(rep["delta"], ref["delta"], rtol=2e-3)
    assert rel_l2(X.cpu().numpy(), ref["X"]) <= TOL_ITER


def test_fft_full_size_ring3d_sampled():
    """512x512x128 with the 31x31x21 template, sampled outputs against the oracle."""
    from paper_1711_11224_gb300 import Plan
    P = synth.ring3d()
    rng = np.random.default_rng(0)
    R = rng.standard_normal(P.Y.shape).astype(np.float32)
    with Plan(P.m, P.p, mode="fft") as pl:
        pl.set_psf(_dev(P.H))
        Y = pl.forward(_dev(P.X_true)).cpu().numpy()
        G = pl.adjoint(_dev(R)).cpu().numpy()
    rng = np.random.default_rng(1)
    si = np.stack([rng.integers(0, s, 1500) for s in Y.shape], axis=1)
    ki = np.stack([rng.integers(0, s, 1500) for s in G.shape], axis=1)
    assert rel_l2(Y[tuple(si.T)], oracle.forward_points(P.X_true, P.H, si)) <= TOL_FFT
    assert rel_l2(G[tuple(ki.T)], oracle.adjoint_points(R, P.H, ki)) <= TOL_FFT

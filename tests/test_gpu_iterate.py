"""GPU parity of the projected-gradient iteration (Steps 1-3) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from _util import TOL_ITER, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _run(P, K, **kw):
    from paper_1711_11224_gb300 import Plan
    with Plan(P.m, P.p) as pl:
        pl.set_psf(_dev(P.H))
        X0 = oracle.x0_crop(P.Y, P.p).astype(np.float32)
        X, rep = pl.iterate(_dev(P.Y), _dev(X0), K=K, **kw)
        return X.cpu().numpy(), rep


def _check(P, K, tol=TOL_ITER, **kw):
    Xg, rep = _run(P, K, **kw)
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), K,
                         delta0=kw.get("delta0"), beta=kw.get("beta", 0.5))
    assert rep["accepted"] == ref["accepted"] == K
    assert rep["status"] == "CDV_OK"
    assert rel_l2(Xg, ref["X"]) <= tol
    np.testing.assert_allclose(rep["f"], ref["f"], rtol=1e-5)
    assert np.all(np.diff(rep["f"]) < 0)                  # the decrease rule of Step 2
    assert np.all(Xg >= 0)
    return Xg, rep, ref


def test_blobs2d_full():
    """64x64, 7x7 Gaussian, 50 iterations (n = 2)."""
    P = synth.blobs2d()
    _check(P, P.K)


def test_fil3d_small_several_tiles():
    """15x15x11 template on a 40x48x36 filament volume: several tiles and ragged tails, 20 iterations."""
    P = synth.scaled_fil3d((40, 48, 36), (15, 15, 11), K=20)
    _check(P, 20)


def test_fil3d_full_100_iterations():
    """256x256x64, 15x15x11 Gaussian, Poisson data, 100 iterations: rel-L2 <= 1e-4 vs FP64."""
    P = synth.fil3d()
    Xg, rep, ref = _check(P, 100)
    assert rep["gmac"] > 0


def test_graph_and_stream_paths_agree_and_repeat():
    P = synth.scaled_fil3d((20, 33, 41), (5, 7, 9), K=10)
    a, ra = _run(P, 10, use_graph=True)
    b, rb = _run(P, 10, use_graph=False)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(ra["f"], rb["f"])
    from paper_1711_11224_gb300 import Plan
    with Plan(P.m, P.p) as pl:                            # replay of the cached graph is deterministic
        pl.set_psf(_dev(P.H))
        X0 = oracle.x0_crop(P.Y, P.p).astype(np.float32)
        Y = _dev(P.Y)
        X = _dev(X0)
        outs = []
        for _ in range(3):
            X.copy_(_dev(X0))
            pl.iterate(Y, X, K=10)
            outs.append(X.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])
    np.testing.assert_array_equal(outs[0], a)


def test_x0_policies():
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((12, 20, 28), (3, 5, 7), K=5)
    with Plan(P.m, P.p) as pl:
        pl.set_psf(_dev(P.H))
        X, rep = pl.iterate(_dev(P.Y), K=0, x0="crop")
        np.testing.assert_array_equal(X.cpu().numpy(), oracle.x0_crop(P.Y, P.p).astype(np.float32))
        assert rep["accepted"] == 0
        np.testing.assert_allclose(rep["f0"], oracle.objective(oracle.x0_crop(P.Y, P.p), P.H, P.Y), rtol=1e-6)
        X, rep = pl.iterate(_dev(P.Y), _dev(np.ones(P.m)), K=3, x0="zero")
        ref = oracle.iterate(P.Y, P.H, np.zeros(P.m), 3)
        assert rel_l2(X.cpu().numpy(), ref["X"]) <= TOL_ITER


def test_backtracking_matches_oracle():
    """delta0 = 8/L forces rejections: the accepted/rejected counts and deltas follow the FP64 rule."""
    P = synth.blobs2d()
    d0 = 8.0 / oracle.lipschitz(P.H)
    Xg, rep = _run(P, 10, delta0=d0, max_rejects=200)     # the oracle has no run-wide cap
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 10, delta0=d0)
    assert rep["accepted"] == ref["accepted"] == 10
    assert rep["rejected"] == ref["rejected"] > 0
    np.testing.assert_allclose(rep["delta"], ref["delta"], rtol=1e-12)
    assert rel_l2(Xg, ref["X"]) <= TOL_ITER


def test_identity_template_converges():
    """H = delta (A = I): the first step reaches max(Y, 0) up to FP32 rounding of the residual."""
    from paper_1711_11224_gb300 import Plan
    rng = np.random.default_rng(1)
    Y = rng.standard_normal((6, 7, 9)).astype(np.float32)
    with Plan((6, 7, 9), (0, 0, 0)) as pl:
        pl.set_psf(_dev(np.ones((1, 1, 1))))
        X, rep = pl.iterate(_dev(Y), _dev(np.full((6, 7, 9), 0.5)), K=5)
    np.testing.assert_allclose(X.cpu().numpy(), np.maximum(Y, 0), rtol=0, atol=4 * 2.0 ** -24 * np.abs(Y).max())
    assert rep["accepted"] >= 1
    assert rep["f"][1] <= 1e-12 * rep["f"][0] + 0.5 * float(np.sum(np.minimum(Y, 0) ** 2)) * (1 + 1e-6)


def test_iterate_host_matches_device():
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((16, 30, 40), (5, 5, 7), K=8)
    X0 = oracle.x0_crop(P.Y, P.p).astype(np.float32)
    a, _ = _run(P, 8)
    with Plan(P.m, P.p) as pl:
        pl.set_psf(_dev(P.H))
        Xh = X0.copy()
        pl.iterate_host(P.Y, Xh, K=8)
    np.testing.assert_array_equal(Xh, a)


def test_richardson_lucy_matches_oracle():
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((14, 26, 30), (5, 7, 5), K=10)
    X0 = np.full(P.m, float(P.Y.mean()), np.float32)
    with Plan(P.m, P.p) as pl:
        pl.set_psf(_dev(P.H))
        X = _dev(X0)
        pl.richardson_lucy(_dev(P.Y), X, 10)
        Xg = X.cpu().numpy()
    ref = oracle.richardson_lucy(P.Y, P.H, X0, 10)
    assert rel_l2(Xg, ref) <= TOL_ITER


@pytest.mark.parametrize("path", ["small", "general"])
def test_blobs2d_both_paths(path):
    """The single-CTA path (whole run in one launch) and the general path both match the oracle."""
    P = synth.blobs2d()
    _check(P, P.K, path=path)


def test_small_path_3d_backtracking_and_policies():
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((4, 16, 24), (3, 5, 7), K=12)
    d0 = 6.0 / oracle.lipschitz(P.H)
    Xs, rs = _run(P, 12, delta0=d0, max_rejects=200, path="small")
    Xg, rg = _run(P, 12, delta0=d0, max_rejects=200, path="general")
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 12, delta0=d0)
    assert rs["accepted"] == rg["accepted"] == ref["accepted"] == 12
    assert rs["rejected"] == rg["rejected"] == ref["rejected"]
    assert rel_l2(Xs, ref["X"]) <= TOL_ITER and rel_l2(Xg, ref["X"]) <= TOL_ITER
    np.testing.assert_allclose(rs["f"], ref["f"], rtol=1e-5)
    assert rs["gmac"] == pytest.approx(rg["gmac"])
    with Plan(P.m, P.p) as pl:
        pl.set_psf(_dev(P.H))
        X, rep = pl.iterate(_dev(P.Y), K=0, x0="crop", path="small")
        np.testing.assert_array_equal(X.cpu().numpy(), oracle.x0_crop(P.Y, P.p).astype(np.float32))
        X, rep = pl.iterate(_dev(P.Y), _dev(np.ones(P.m)), K=3, x0="zero", path="small")
        assert rel_l2(X.cpu().numpy(), oracle.iterate(P.Y, P.H, np.zeros(P.m), 3)["X"]) <= TOL_ITER


def test_small_path_rejects_large_problem():
    from paper_1711_11224_gb300 import CdvError, Plan
    with Plan((64, 64, 64), (1, 1, 1)) as pl:
        pl.set_psf(_dev(np.ones((3, 3, 3)) / 27))
        with pytest.raises(CdvError, match="UNSUPPORTED"):
            pl.iterate(_dev(np.zeros((66, 66, 66))), K=1, path="small")


def test_resume_equals_uninterrupted_run():
    """Checkpoint/resume: K1 steps, then K - K1 more from the saved iterate, equal K steps at once."""
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((10, 40, 36), (5, 7, 9), K=12)
    with Plan(P.m, P.p) as pl:
        pl.set_psf(_dev(P.H))
        Y = _dev(P.Y)
        Xa, ra = pl.iterate(Y, K=12, x0="crop", path="general")
        Xb, rb1 = pl.iterate(Y, K=5, x0="crop", path="general")
        ckpt = Xb.cpu().numpy()                                   # the whole iteration state at a fixed step rule
        Xc, rb2 = pl.iterate(Y, _dev(ckpt), K=7, x0="given", path="general")
    np.testing.assert_array_equal(Xa.cpu().numpy(), Xc.cpu().numpy())
    np.testing.assert_array_equal(ra["f"][5:], rb2["f"])


@pytest.mark.parametrize("lam,sigma", [(0.05, 0.0), (0.0, 0.3), (0.05, 0.1)])
def test_tikhonov_armijo_match_oracle(lam, sigma):
    """The Tikhonov term (gradient + lambda x, f + lambda/2 ||x||^2) and the Armijo condition on the
    general path (several CTAs, stream and graph launches) against the FP64 oracle."""
    P = synth.scaled_fil3d((12, 60, 50), (5, 5, 7), K=12)
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 12, tikhonov=lam, armijo=sigma)
    for g in (True, False):
        Xg, rep = _run(P, 12, tikhonov=lam, armijo=sigma, use_graph=g)
        assert rep["accepted"] == ref["accepted"] == 12 and rep["status"] == "CDV_OK"
        assert rep["rejected"] == ref["rejected"]
        np.testing.assert_allclose(rep["delta"], ref["delta"], rtol=1e-12)
        np.testing.assert_allclose(rep["f"], ref["f"], rtol=1e-5)
        assert rel_l2(Xg, ref["X"]) <= TOL_ITER


@pytest.mark.parametrize("sigma,delta,rejected", [(0.4, 1.0, 0), (0.6, 0.5, 1)])
def test_armijo_identity_template_closed_form(sigma, delta, rejected):
    """H = delta, x_0 = 0, y_c > 0: the full step passes the Armijo test for sigma < 1/2 only."""
    from paper_1711_11224_gb300 import Plan
    rng = np.random.default_rng(12)
    Y = (rng.random((6, 8)) + 0.5).astype(np.float32)
    H = np.zeros((3, 3))
    H[1, 1] = 1.0
    with Plan((4, 6), (1, 1)) as pl:
        pl.set_psf(_dev(H))
        X, rep = pl.iterate(_dev(Y), _dev(np.zeros((4, 6))), K=1, armijo=sigma, path="general")
    assert rep["accepted"] == 1 and rep["rejected"] == rejected
    assert rep["delta"][0] == delta
    np.testing.assert_array_equal(X.cpu().numpy(), np.float32(delta) * Y[1:-1, 1:-1])


def test_step_variants_rejected_where_unsupported():
    from paper_1711_11224_gb300 import BatchPlan, CdvError, Plan
    P = synth.blobs2d()
    with Plan(P.m, P.p) as pl:
        pl.set_psf(_dev(P.H))
        with pytest.raises(CdvError, match="UNSUPPORTED"):
            pl.iterate(_dev(P.Y), K=2, path="small", tikhonov=0.1)
        X, rep = pl.iterate(_dev(P.Y), K=2, tikhonov=0.1)          # auto: runs on the general path
        assert rep["accepted"] == 2
        with pytest.raises(CdvError, match="INVALID_ARG"):
            pl.iterate(_dev(P.Y), K=2, armijo=1.0)
        with pytest.raises(CdvError, match="UNSUPPORTED"):
            pl.iterate(_dev(P.Y), K=2, path="small", bb=True)
    with BatchPlan([P.m], [P.p], autotune=False) as bp:
        bp.set_psfs([_dev(P.H)])
        with pytest.raises(CdvError, match="UNSUPPORTED"):
            bp.iterate([_dev(P.Y)], K=2, armijo=0.1)


@pytest.mark.parametrize("kw", [{"bb": True}, {"bb": True, "tikhonov": 0.05, "armijo": 1e-4}])
def test_bb_matches_oracle(kw):
    """Barzilai-Borwein first trials (lagged by one step) against the FP64 oracle: the same accepted and
    rejected trials; the lengths <s,s>/<s,v> agree to 2e-3 (v is a difference of FP32 gradients that
    cancels to about 1e-3 of their size, so its relative error is about 1e-4)."""
    P = synth.scaled_fil3d((12, 60, 50), (5, 5, 7), K=20)
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 20, **kw)
    Xg, rep = _run(P, 20, max_rejects=200, **kw)            # the oracle has no run-wide reject cap
    assert rep["accepted"] == ref["accepted"] == 20 and rep["status"] == "CDV_OK"
    assert rep["rejected"] == ref["rejected"] > 0
    np.testing.assert_allclose(rep["delta"], ref["delta"], rtol=2e-3)
    assert np.max(ref["delta"]) * (oracle.lipschitz(P.H) + kw.get("tikhonov", 0.0)) > 4   # long steps taken
    np.testing.assert_allclose(rep["f"], ref["f"], rtol=1e-4)
    assert rel_l2(Xg, ref["X"]) <= TOL_ITER

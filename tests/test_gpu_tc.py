"""Tensor-core (tcgen05) forms against the FP64 oracle.

split-BF16x3 is held to the FP32 bar (relative L2 <= 1e-5 per convolution);
BF16 and TF32 products are reported against bounds derived from their unit
roundoff (BF16 2^-9, TF32 2^-12 relative per input, averaged over the taps).
Integer data are exact in every mode: products and partial sums of small
integers are representable in BF16/TF32 and FP32.
"""
import numpy as np
import pytest

import oracle
import synth
from _util import TOL_CONV, TOL_ITER, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"split3": TOL_CONV, "tf32": 1e-3, "bf16": 8e-3}
MODES = ["split3", "tf32", "bf16"]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _plan(m, q, mode):
    from paper_1711_11224_gb300 import Plan
    return Plan(m, [(v - 1) // 2 for v in q], mode=mode)


SHAPES = [
    ((3, 130, 40), (3, 5, 7)),        # two row tiles, ragged columns
    ((4, 200, 148), (3, 7, 21)),      # 11 column tiles
    ((2, 90, 33), (3, 31, 9)),        # 31 template rows
    ((3, 20, 300), (1, 3, 5)),        # output rows wider than one CTA (two column groups)
    ((50, 70), (7, 7)),               # n = 2
    ((3, 4, 5), (7, 9, 11)),          # template larger than the volume
    ((60, 400, 300), (3, 5, 7)),      # 320 forward tiles: several tiles per persistent CTA
]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("m,q", SHAPES)
def test_tc_forward_adjoint(mode, m, q):
    X, H, R = synth.random_case(m, q, seed=3)
    with _plan(m, q, mode) as pl:
        pl.set_psf(_dev(H))
        Y = pl.forward(_dev(X)).cpu().numpy()
        G = pl.adjoint(_dev(R)).cpu().numpy()
        pl.sync()
    assert rel_l2(Y, oracle.forward(X, H)) <= TOL[mode]
    assert rel_l2(G, oracle.adjoint(R, H)) <= TOL[mode]


@pytest.mark.parametrize("mode", MODES)
def test_tc_integer_exact(mode):
    m, q = (4, 140, 60), (3, 5, 9)
    X, H = synth.integer_case(m, q, seed=4)
    rng = np.random.default_rng(1)
    R = rng.integers(-4, 5, size=tuple(a + b - 1 for a, b in zip(m, q))).astype(np.float32)
    with _plan(m, q, mode) as pl:
        pl.set_psf(_dev(H))
        Y = pl.forward(_dev(X)).cpu().numpy()
        G = pl.adjoint(_dev(R)).cpu().numpy()
    np.testing.assert_array_equal(Y.astype(np.float64), oracle.forward(X, H))
    np.testing.assert_array_equal(G.astype(np.float64), oracle.adjoint(R, H))


@pytest.mark.parametrize("mode", ["split3", "tf32"])
def test_tc_iterate(mode):
    """Steps 1-3 on the tensor cores: split-BF16x3 within the FP32 iteration bar after 20 steps."""
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((24, 140, 50), (7, 9, 11), K=20)
    with Plan(P.m, P.p, mode=mode) as pl:
        pl.set_psf(_dev(P.H))
        X, rep = pl.iterate(_dev(P.Y), K=20, x0="crop")
        Xg = X.cpu().numpy()
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 20)
    assert rep["accepted"] == 20 and rep["status"] == "CDV_OK"
    assert np.all(np.diff(rep["f"]) < 0)
    tol = TOL_ITER if mode == "split3" else 5e-3
    assert rel_l2(Xg, ref["X"]) <= tol
    # f = 1/2 ||Ax - y||^2: the residual cancels, so its relative error exceeds the per-convolution one
    np.testing.assert_allclose(rep["f"], ref["f"], rtol=1e-4 if mode == "split3" else 2e-3)


@pytest.mark.parametrize("mode", ["split3", "tf32"])
def test_tc_tikhonov_armijo(mode):
    """Tikhonov term and Armijo condition fused into the tensor-core epilogues, against the oracle."""
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((20, 140, 50), (7, 9, 11), K=10)
    lam, sigma = 0.05, 0.1
    with Plan(P.m, P.p, mode=mode) as pl:
        pl.set_psf(_dev(P.H))
        X, rep = pl.iterate(_dev(P.Y), K=10, x0="crop", tikhonov=lam, armijo=sigma)
        Xg = X.cpu().numpy()
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 10, tikhonov=lam, armijo=sigma)
    assert rep["accepted"] == ref["accepted"] == 10 and rep["status"] == "CDV_OK"
    np.testing.assert_allclose(rep["delta"], ref["delta"], rtol=1e-12)
    assert rel_l2(Xg, ref["X"]) <= (TOL_ITER if mode == "split3" else 5e-3)
    np.testing.assert_allclose(rep["f"], ref["f"], rtol=1e-4 if mode == "split3" else 2e-3)


def test_tc_bb():
    """Barzilai-Borwein first trials with the tensor-core epilogues (split-BF16x3) against the oracle."""
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((20, 140, 50), (7, 9, 11), K=20)
    with Plan(P.m, P.p, mode="split3") as pl:
        pl.set_psf(_dev(P.H))
        X, rep = pl.iterate(_dev(P.Y), K=20, x0="crop", bb=True, max_rejects=200)
        Xg = X.cpu().numpy()
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 20, bb=True)
    assert rep["accepted"] == ref["accepted"] == 20 and rep["rejected"] == ref["rejected"]
    np.testing.assert_allclose(rep["delta"], ref["delta"], rtol=2e-3)
    assert rel_l2(Xg, ref["X"]) <= TOL_ITER
    np.testing.assert_allclose(rep["f"], ref["f"], rtol=1e-4)


def test_tc_iterate_many_tiles():
    """More output tiles than SMs, so each persistent CTA carries its rings across tiles."""
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((40, 300, 260), (5, 5, 7), K=5)
    with Plan(P.m, P.p, mode="split3") as pl:
        pl.set_psf(_dev(P.H))
        X, rep = pl.iterate(_dev(P.Y), K=5, x0="crop")
        Xg = X.cpu().numpy()
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 5)
    assert rep["accepted"] == 5 and rep["status"] == "CDV_OK"
    assert rel_l2(Xg, ref["X"]) <= TOL_ITER
    np.testing.assert_allclose(rep["f"], ref["f"], rtol=1e-4)


def test_tc_graph_matches_stream():
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((10, 140, 40), (5, 5, 7), K=6)
    outs = []
    for g in (True, False):
        with Plan(P.m, P.p, mode="split3") as pl:
            pl.set_psf(_dev(P.H))
            X, _ = pl.iterate(_dev(P.Y), K=6, x0="crop", use_graph=g)
            outs.append(X.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])


def test_tc_full_size_ring3d_sampled():
    """512x512x128 with the 31x31x21 template in split-BF16x3, sampled outputs against the oracle."""
    P = synth.ring3d()
    rng = np.random.default_rng(0)
    R = rng.standard_normal(P.Y.shape).astype(np.float32)
    with _plan(P.m, P.H.shape, "split3") as pl:
        pl.set_psf(_dev(P.H))
        Y = pl.forward(_dev(P.X_true)).cpu().numpy()
        G = pl.adjoint(_dev(R)).cpu().numpy()
    rng = np.random.default_rng(1)
    si = np.stack([rng.integers(0, s, 1500) for s in Y.shape], axis=1)
    ki = np.stack([rng.integers(0, s, 1500) for s in G.shape], axis=1)
    assert rel_l2(Y[tuple(si.T)], oracle.forward_points(P.X_true, P.H, si)) <= TOL_CONV
    assert rel_l2(G[tuple(ki.T)], oracle.adjoint_points(R, P.H, ki)) <= TOL_CONV


def test_tc_rl_is_fp32_only():
    from paper_1711_11224_gb300 import CdvError
    with _plan((4, 20, 20), (3, 3, 3), "bf16") as pl:
        pl.set_psf(_dev(np.ones((3, 3, 3)) / 27))
        with pytest.raises(CdvError, match="UNSUPPORTED"):
            pl.richardson_lucy(_dev(np.ones((6, 22, 22))), _dev(np.ones((4, 20, 20))), 2)


@pytest.mark.parametrize("mode", ["split3", "bf16", "tf32"])
def test_tc_describe_counts_the_kernel_loops(mode, monkeypatch):
    """Executed MACs the library reports for the wide kernel, recounted here from the tiling it reports."""
    monkeypatch.setenv("CDV_TC_KERNEL", "wide")
    m, q = (40, 300, 130), (31, 31, 21)
    p = [(v - 1) // 2 for v in q]
    with _plan(m, q, mode) as pl:
        info = pl.describe()
    ept = 4 if mode == "tf32" else 8
    nprod = 3 if mode == "split3" else 1
    assert info["algorithmic_macs"] == float(np.prod(m) * np.prod(q))
    for d in (0, 1):
        a = m if d == 0 else tuple(x + 2 * y for x, y in zip(m, p))
        b = tuple(x + 2 * y for x, y in zip(m, p)) if d == 0 else m
        o = (0, 0, 0) if d == 0 else tuple(2 * y for y in p)
        W = info["cols"][d]
        assert W in (8, 16)
        e = (o[2] - (q[2] - 1)) % ept
        K = -(-(e + q[2] + W - 1) // 16) * 16
        assert info["K"][d] == K
        P = 128 // W
        n_sum = 0
        for S1 in range(0, b[0], P):
            s1_end = min(S1 + P, b[0])
            for u in range(max(0, S1 + o[0] - q[0] + 1), min(a[0] - 1, s1_end - 1 + o[0]) + 1):
                planes = [i for i in range(s1_end - S1) if 0 <= S1 + i + o[0] - u < q[0]]
                nv = len(planes) + (1 if W == 8 and len(planes) % 2 else 0)
                n_sum += W * nv
        mtiles = sum(min(2, -(-(b[1] - S2) // 128)) for S2 in range(0, b[1], 256))
        tiles3 = -(-b[2] // W)
        assert info["tiles"][d] == -(-b[0] // P) * -(-b[1] // 256) * tiles3
        expect = n_sum * mtiles * 128 * K * q[1] * tiles3 * nprod
        assert info["executed_macs"][d] == pytest.approx(expect, rel=1e-12)
    # the 21-wide contiguous axis takes 8 columns per plane (K = 32 rather than 48)
    assert info["cols"] == [8, 8]

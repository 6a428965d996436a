"""The narrow tensor-core kernel (4 output columns, 32 sliding plane slots) against the FP64 oracle.

CDV_TC_KERNEL=narrow makes every plan whose template allows it (BF16 forms,
q1 <= 31, windows that start on 4-column boundaries: q3 = 1 mod 4) run both
directions on it; the shapes below cover ragged column groups of both shadow
copies, several plane chunks per volume, several row blocks, one-plane and
one-row volumes, templates larger than the volume, odd and even numbers of
window chunks per template row (paired across rows when odd), the
iteration's epilogues with and without the step-rule variants, re-tried
trials that reuse the stored gradient, and the graph against the stream.
"""
import numpy as np
import pytest

import oracle
import synth
from _util import TOL_CONV, TOL_ITER, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"split3": TOL_CONV, "bf16": 8e-3}


@pytest.fixture(autouse=True, params=["narrow_rows", "narrow_flat"])
def narrow(monkeypatch, request):
    """Both layouts of the forward's M dimension: rows of one column group, or (column group, row)."""
    monkeypatch.setenv("CDV_TC_KERNEL", request.param)
    return request.param


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _plan(m, q, mode):
    from paper_1711_11224_gb300 import Plan
    pl = Plan(m, [(v - 1) // 2 for v in q], mode=mode)
    assert pl.describe()["cols"] == [4, 4]
    return pl


SHAPES = [
    ((40, 20, 24), (9, 5, 13)),        # 2 chunks per template row
    ((40, 20, 30), (31, 7, 21)),       # 3 chunks per row (paired across rows), 31 template planes
    ((70, 9, 17), (31, 3, 21)),        # several plane chunks
    ((5, 270, 12), (7, 31, 5)),        # two row blocks, 1 chunk per row
    ((3, 4, 5), (7, 9, 21)),           # template larger than the volume
    ((1, 33, 41), (1, 5, 9)),          # one plane, one template plane
    ((64, 130, 37), (5, 3, 13)),       # ragged rows and columns, 64 planes
    ((100, 1, 50), (21, 1, 21)),       # one row
]


@pytest.mark.parametrize("mode", ["split3", "bf16"])
@pytest.mark.parametrize("m,q", SHAPES)
def test_narrow_forward_adjoint(mode, m, q):
    X, H, R = synth.random_case(m, q, seed=5)
    with _plan(m, q, mode) as pl:
        pl.set_psf(_dev(H))
        Y = pl.forward(_dev(X)).cpu().numpy()
        G = pl.adjoint(_dev(R)).cpu().numpy()
        pl.sync()
    assert rel_l2(Y, oracle.forward(X, H)) <= TOL[mode]
    assert rel_l2(G, oracle.adjoint(R, H)) <= TOL[mode]


@pytest.mark.parametrize("mode", ["split3", "bf16"])
def test_narrow_integer_exact(mode):
    m, q = (36, 140, 45), (7, 5, 13)
    X, H = synth.integer_case(m, q, seed=6)
    rng = np.random.default_rng(2)
    R = rng.integers(-4, 5, size=tuple(a + b - 1 for a, b in zip(m, q))).astype(np.float32)
    with _plan(m, q, mode) as pl:
        pl.set_psf(_dev(H))
        Y = pl.forward(_dev(X)).cpu().numpy()
        G = pl.adjoint(_dev(R)).cpu().numpy()
    np.testing.assert_array_equal(Y.astype(np.float64), oracle.forward(X, H))
    np.testing.assert_array_equal(G.astype(np.float64), oracle.adjoint(R, H))


def test_narrow_iterate_matches_oracle():
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((40, 140, 50), (9, 9, 13), K=20)
    with Plan(P.m, P.p, mode="split3") as pl:
        assert pl.describe()["cols"] == [4, 4]
        pl.set_psf(_dev(P.H))
        X, rep = pl.iterate(_dev(P.Y), K=20, x0="crop")
        Xg = X.cpu().numpy()
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 20)
    assert rep["accepted"] == 20 and rep["status"] == "CDV_OK"
    assert rel_l2(Xg, ref["X"]) <= TOL_ITER
    np.testing.assert_allclose(rep["f"], ref["f"], rtol=1e-4)


def test_narrow_backtracking_reuses_gradient():
    """A first trial of 8/L is rejected and halved (the re-tried trials reuse the stored gradient)."""
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((20, 90, 40), (5, 5, 9), K=6)
    d0 = 8.0 / oracle.lipschitz(P.H)
    with Plan(P.m, P.p, mode="split3") as pl:
        pl.set_psf(_dev(P.H))
        X, rep = pl.iterate(_dev(P.Y), K=6, x0="crop", delta0=d0, max_rejects=200)
        Xg = X.cpu().numpy()
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 6, delta0=d0)
    assert ref["rejected"] > 0
    assert rep["accepted"] == ref["accepted"] == 6 and rep["rejected"] == ref["rejected"]
    np.testing.assert_allclose(rep["delta"], ref["delta"], rtol=1e-12)
    assert rel_l2(Xg, ref["X"]) <= TOL_ITER


def test_narrow_variants_match_oracle():
    """Tikhonov term, Armijo condition and Barzilai-Borwein lengths in the narrow kernel's epilogue."""
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((20, 140, 50), (7, 9, 13), K=12)
    with Plan(P.m, P.p, mode="split3") as pl:
        pl.set_psf(_dev(P.H))
        X, rep = pl.iterate(_dev(P.Y), K=12, x0="crop", tikhonov=0.05, armijo=0.1)
        Xa = X.cpu().numpy()
        X, rb = pl.iterate(_dev(P.Y), K=12, x0="crop", bb=True, max_rejects=200)
        Xb = X.cpu().numpy()
    ra = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 12, tikhonov=0.05, armijo=0.1)
    rbo = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 12, bb=True)
    assert rep["accepted"] == ra["accepted"] == 12
    assert rel_l2(Xa, ra["X"]) <= TOL_ITER
    assert rb["accepted"] == rbo["accepted"] == 12 and rb["rejected"] == rbo["rejected"]
    np.testing.assert_allclose(rb["delta"], rbo["delta"], rtol=2e-3)
    assert rel_l2(Xb, rbo["X"]) <= TOL_ITER


def test_narrow_graph_matches_stream():
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((40, 140, 40), (5, 5, 9), K=6)
    outs = []
    for g in (True, False):
        with Plan(P.m, P.p, mode="split3") as pl:
            pl.set_psf(_dev(P.H))
            X, _ = pl.iterate(_dev(P.Y), K=6, x0="crop", use_graph=g)
            outs.append(X.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])


def _narrow_bounds(m, q, d):
    """Bounds on the narrow kernel's MMA work (rows layout) whatever the cut of the output planes into
    32-aligned ranges: at least 4 columns per (input plane, output plane) pair it joins, at most N = 128
    for every input plane of every range with the finest cut (the most input planes)."""
    p = [(v - 1) // 2 for v in q]
    kc = -(-(q[2] + 3) // 8)
    steps = -(-(q[1] * kc) // 2)
    a = m if d == 0 else tuple(x + 2 * y for x, y in zip(m, p))
    b = tuple(x + 2 * y for x, y in zip(m, p)) if d == 0 else m
    o = (0, 0, 0) if d == 0 else tuple(2 * y for y in p)
    pairs = sum(1 for s in range(b[0]) for j in range(q[0]) if 0 <= s + o[0] - j < a[0])
    planes = 0
    for S1 in range(0, b[0], 32):
        s1_end = min(S1 + 32, b[0])
        planes += min(a[0] - 1, s1_end - 1 + o[0]) - max(0, S1 + o[0] - q[0] + 1) + 1
    unit = 128 * 16 * steps * 3 * sum(min(2, -(-(b[1] - S2) // 128)) for S2 in range(0, b[1], 256)) * -(-b[2] // 4)
    return 4 * pairs * unit, 128 * planes * unit, b


def test_narrow_describe_counts_the_kernel_loops(narrow):
    """Executed MACs the library reports for the narrow kernel (rows layout) lie within the bounds of its
    loops for any cut of the planes, and are a whole number of its MMAs."""
    if narrow != "narrow_rows":
        pytest.skip("counted for the rows layout")
    m, q = (40, 300, 130), (31, 31, 21)
    with _plan(m, q, "split3") as pl:
        info = pl.describe()
    kc = -(-(q[2] + 3) // 8)
    assert info["K"] == [8 * kc, 8 * kc]
    for d in (0, 1):
        lo, hi, b = _narrow_bounds(m, q, d)
        assert lo <= info["executed_macs"][d] <= hi
        assert info["executed_macs"][d] % (16 * 128 * 16 * 3) == 0
        assert info["tiles"][d] >= -(-b[1] // 256) * -(-b[2] // 4)

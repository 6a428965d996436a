"""Failure paths that the device reports without faulting.

* Non-finite objective: a NaN in Y makes f(x_0) NaN; a huge first step length
  makes the first trial's residual overflow FP32 (f = inf).  Both end the run
  with CDV_ERR_NONFINITE and leave X at the last accepted (finite) iterate, on
  the CUDA-graph path, the stream path, the single-CTA path and the tensor-core
  path.
* Timed-out waits: the tensor-core kernels bound every barrier wait; with a
  budget of one clock cycle the waits run out, the kernel records
  CDV_ERR_TIMEOUT, drains its own copies and exits, and the plan works again
  once the status has been read and the budget restored.
* Idle budget of the persistent batched run: with one clock cycle a CTA that
  finds no tile at once records CDV_ERR_TIMEOUT, every CTA leaves, the call
  reports it, and the next run with the default budget is exact.
"""
import numpy as np
import pytest

import oracle
import synth
from _util import TOL_CONV, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT = 6


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


CASES = [  # (mode, path, use_graph)
    ("fp32", "general", True), ("fp32", "general", False), ("fp32", "small", True), ("split3", "general", True),
]


@pytest.mark.parametrize("mode,path,graph", CASES)
def test_nan_in_y_is_nonfinite(mode, path, graph):
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((4, 24, 40), (3, 3, 5), K=5) if path != "small" else synth.blobs2d()
    Y = P.Y.copy()
    Y.flat[Y.size // 3] = np.nan
    X0 = np.maximum(P.Y[tuple(slice(p, p + m) for p, m in zip(P.p, P.m))], 0).astype(np.float32)
    with Plan(P.m, P.p, mode=mode) as pl:
        pl.set_psf(_dev(P.H))
        X = _dev(X0)
        X, rep = pl.iterate(_dev(Y), X, K=5, x0="given", path=path, use_graph=graph)
        Xh = X.cpu().numpy()
    assert rep["status"] == "CDV_ERR_NONFINITE" and rep["accepted"] == 0
    assert not np.isfinite(rep["f0"])
    np.testing.assert_array_equal(Xh, X0)


@pytest.mark.parametrize("mode,path,graph", CASES)
def test_trial_overflow_is_nonfinite(mode, path, graph):
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((4, 24, 40), (3, 3, 5), K=5) if path != "small" else synth.blobs2d()
    X0 = np.maximum(P.Y[tuple(slice(p, p + m) for p, m in zip(P.p, P.m))], 0).astype(np.float32)
    with Plan(P.m, P.p, mode=mode) as pl:
        pl.set_psf(_dev(P.H))
        X = _dev(X0)
        # a first step of 1e30: the trial's residual is about 1e30 and its square overflows FP32
        X, rep = pl.iterate(_dev(P.Y), X, K=5, x0="given", path=path, use_graph=graph, delta0=1e30,
                            max_halvings=0)
        Xh = X.cpu().numpy()
    assert np.isfinite(rep["f0"])
    assert rep["status"] == "CDV_ERR_NONFINITE" and rep["accepted"] == 0
    np.testing.assert_array_equal(Xh, X0)


def test_tc_wait_budget_runs_out_and_recovers():
    from paper_1711_11224_gb300 import CdvError, Plan
    m, q = (6, 140, 40), (3, 5, 7)
    X, H, R = synth.random_case(m, q, seed=5)
    with Plan(m, [(v - 1) // 2 for v in q], mode="split3") as pl:
        pl.set_psf(_dev(H))
        pl.set_wait_cycles(1)
        pl.forward(_dev(X))
        with pytest.raises(CdvError) as ei:
            pl.sync()
        assert ei.value.status == TIMEOUT
        pl.set_wait_cycles(0)                            # the default budget again
        Y = pl.forward(_dev(X)).cpu().numpy()
        pl.sync()
        assert rel_l2(Y, oracle.forward(X, H)) <= TOL_CONV


def test_tc_iterate_timeout_reported_then_cleared():
    from paper_1711_11224_gb300 import Plan
    P = synth.scaled_fil3d((8, 140, 40), (3, 5, 7), K=4)
    with Plan(P.m, P.p, mode="split3") as pl:
        pl.set_psf(_dev(P.H))
        pl.set_wait_cycles(1)
        _, rep = pl.iterate(_dev(P.Y), K=4, x0="crop")
        assert rep["status"] == "CDV_ERR_TIMEOUT"
        pl.set_wait_cycles(0)
        X, rep = pl.iterate(_dev(P.Y), K=4, x0="crop")      # the report above cleared the status word
        Xg = X.cpu().numpy()
        pl.sync()
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 4)
    assert rep["status"] == "CDV_OK" and rep["accepted"] == 4
    assert rel_l2(Xg, ref["X"]) <= 1e-4


def test_batch_persistent_idle_budget_runs_out_and_recovers():
    """A one-cycle idle budget: CTAs that find no tile at once record CDV_ERR_TIMEOUT and every CTA
    leaves; the call reports it, and the next run with the default budget is exact again."""
    from paper_1711_11224_gb300 import BatchPlan, CdvError
    probs = [synth.scaled_fil3d(m, q, seed=i, K=3) for i, (m, q) in
             enumerate([((8, 40, 33), (3, 5, 7)), ((12, 30, 40), (5, 5, 7))])]
    with BatchPlan([P.m for P in probs], [P.p for P in probs], autotune=False) as bp:
        bp.set_psfs([_dev(P.H) for P in probs])
        Ys = [_dev(P.Y) for P in probs]
        bp.set_wait_cycles(1)
        with pytest.raises(CdvError) as ei:
            bp.iterate(Ys, K=3, x0="crop")
        assert ei.value.status == TIMEOUT
        bp.set_wait_cycles(0)
        Xs, reps = bp.iterate(Ys, K=3, x0="crop")
        Xb = [X.cpu().numpy() for X in Xs]
        Xs2, _ = bp.iterate(Ys, K=3, x0="crop", path="general")
        for a, X in zip(Xb, Xs2):
            np.testing.assert_array_equal(a, X.cpu().numpy())
    assert all(r["status"] == "CDV_OK" and r["accepted"] == 3 for r in reps)

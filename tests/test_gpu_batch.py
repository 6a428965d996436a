"""Batched solver: many uneven volumes with their own templates iterated together.

A volume's iterates do not depend on the tile shape nor on the other volumes,
nor on how the run is launched (one persistent launch, the default, or common
trial slots of batched launches), so the batched result must equal
cdv_iterate on each volume alone, bit for bit; cdv_iterate itself is held to
the FP64 oracle elsewhere, and here too on two small volumes and, after 200
steps, on five volumes of the 64-volume workload.
"""
import numpy as np
import pytest

import oracle
import synth
from _util import TOL_ITER, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [((12, 30, 40), (5, 5, 7)), ((8, 50, 33), (3, 7, 9)), ((20, 20, 20), (7, 3, 5)),
          ((6, 64, 17), (3, 5, 7)), ((16, 16, 64), (1, 3, 11))]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _problems(shapes, K):
    return [synth.scaled_fil3d(m, q, seed=i, K=K) for i, (m, q) in enumerate(shapes)]


def _single(P, K, **kw):
    from paper_1711_11224_gb300 import Plan
    with Plan(P.m, P.p) as pl:
        pl.set_psf(_dev(P.H))
        X, rep = pl.iterate(_dev(P.Y), K=K, x0="crop", path="general", **kw)
        return X.cpu().numpy(), rep


@pytest.mark.parametrize("path", ["persistent", "general"])
@pytest.mark.parametrize("autotune", [True, False])
def test_batch_equals_single_volume_runs(autotune, path):
    from paper_1711_11224_gb300 import BatchPlan
    K = 8
    probs = _problems(SHAPES, K)
    with BatchPlan([P.m for P in probs], [P.p for P in probs], autotune=autotune) as bp:
        bp.set_psfs([_dev(P.H) for P in probs])
        Xs, reps = bp.iterate([_dev(P.Y) for P in probs], K=K, x0="crop", path=path)
        Xb = [X.cpu().numpy() for X in Xs]
    for P, X, r in zip(probs, Xb, reps):
        Xs_, rs = _single(P, K)
        assert r["accepted"] == rs["accepted"] == K and r["status"] == "CDV_OK"
        np.testing.assert_array_equal(X, Xs_)
        np.testing.assert_allclose(r["f"], rs["f"], rtol=1e-12)


def test_batch_matches_oracle():
    from paper_1711_11224_gb300 import BatchPlan
    probs = _problems(SHAPES[:2], 10)
    with BatchPlan([P.m for P in probs], [P.p for P in probs]) as bp:
        bp.set_psfs([_dev(P.H) for P in probs])
        Xs, reps = bp.iterate([_dev(P.Y) for P in probs], K=10, x0="crop")
    for P, X, r in zip(probs, Xs, reps):
        ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 10)
        assert r["accepted"] == ref["accepted"] == 10
        assert rel_l2(X.cpu().numpy(), ref["X"]) <= TOL_ITER
        np.testing.assert_allclose(r["f"], ref["f"], rtol=1e-5)


def test_batch_graph_replay_and_repeat():
    """Graph replays, stream launches and both paths, switched back and forth on one plan, agree."""
    from paper_1711_11224_gb300 import BatchPlan
    probs = _problems(SHAPES[:3], 5)
    with BatchPlan([P.m for P in probs], [P.p for P in probs]) as bp:
        bp.set_psfs([_dev(P.H) for P in probs])
        Ys = [_dev(P.Y) for P in probs]
        Xs = [torch.empty(P.m, device="cuda") for P in probs]
        outs = []
        for g, path in ((True, "persistent"), (True, "persistent"), (False, "persistent"), (True, "general"),
                        (False, "general"), (True, "persistent")):
            bp.iterate(Ys, Xs, K=5, x0="crop", use_graph=g, path=path)
            outs.append([X.cpu().numpy() for X in Xs])
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            np.testing.assert_array_equal(a, b)


def test_batch_backtracking_and_early_stop():
    """Rejected trials (a first length of 8/L halved back) and volumes that stop at different times
    (when they exceed max_rejects) in the persistent run, against the slot path."""
    from paper_1711_11224_gb300 import BatchPlan
    probs = _problems(SHAPES[:4], 6)
    res = {}
    with BatchPlan([P.m for P in probs], [P.p for P in probs]) as bp:
        bp.set_psfs([_dev(P.H) for P in probs])
        for path in ("persistent", "general"):
            Xs, reps = bp.iterate([_dev(P.Y) for P in probs], K=6, x0="crop", delta0=8.0 / max(
                oracle.lipschitz(P.H) for P in probs), max_rejects=3, path=path)
            res[path] = ([X.cpu().numpy() for X in Xs], reps)
    (Xp, rp), (Xg, rg) = res["persistent"], res["general"]
    assert any(r["rejected"] > 0 for r in rp)
    for a, b, r1, r2 in zip(Xp, Xg, rp, rg):
        np.testing.assert_array_equal(a, b)
        assert (r1["accepted"], r1["rejected"], r1["status"]) == (r2["accepted"], r2["rejected"], r2["status"])


def test_batch_small_path_rejected():
    from paper_1711_11224_gb300 import BatchPlan, _binding
    probs = _problems(SHAPES[:2], 2)
    with BatchPlan([P.m for P in probs], [P.p for P in probs], autotune=False) as bp:
        bp.set_psfs([_dev(P.H) for P in probs])
        with pytest.raises(_binding.CdvError, match="UNSUPPORTED"):
            bp.iterate([_dev(P.Y) for P in probs], K=2, x0="crop", path="small")


@pytest.fixture(scope="module")
def batch64_run():
    """64 uneven volumes (sizes U[32,256]^2 x U[16,128], templates odd U[5,21]), 200 steps, one graph."""
    from paper_1711_11224_gb300 import BatchPlan
    probs = synth.batch64(K=200)
    with BatchPlan([P.m for P in probs], [P.p for P in probs]) as bp:
        bp.set_psfs([_dev(P.H) for P in probs])
        Xs, reps = bp.iterate([_dev(P.Y) for P in probs], K=200, x0="crop")
        Xh = [X.cpu().numpy() for X in Xs]
    return probs, Xh, reps


def test_batch64_workload_subset_equals_single(batch64_run):
    probs, Xs, reps = batch64_run
    assert all(r["status"] == "CDV_OK" and r["accepted"] == 200 for r in reps)
    assert all(np.all(np.diff(r["f"]) < 0) for r in reps)
    for i in (0, 17, 40, 63):
        Xs_, rs = _single(probs[i], 200)
        np.testing.assert_array_equal(Xs[i], Xs_)


# The cheapest volumes of the batch for the FP64 oracle, two of them with a 21-wide template axis
# (volume 48: 48x86x32 with 7x21x15; volume 63: 65x72x61 with 15x7x21 along the contiguous axis).
ORACLE_VOLUMES = (19, 13, 43, 48, 63)


def test_batch64_volumes_match_oracle_200_steps(batch64_run):
    """200 accepted steps of the batched solver against the oracle's 200 steps on the same volume."""
    probs, Xs, reps = batch64_run
    assert any(21 in probs[i].H.shape for i in ORACLE_VOLUMES)
    assert probs[63].H.shape[2] == 21
    for i in ORACLE_VOLUMES:
        P = probs[i]
        ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), 200)
        assert ref["accepted"] == reps[i]["accepted"] == 200
        e = rel_l2(Xs[i], ref["X"])
        print("volume %d m=%s q=%s: x_200 rel-L2 %.3e" % (i, P.m, P.H.shape, e))
        assert e <= TOL_ITER
        np.testing.assert_allclose(reps[i]["f"], ref["f"], rtol=1e-5)


def test_single_plan_rejects_the_persistent_path():
    """CDV_PATH_PERSISTENT belongs to the batched solver; cdv_iterate answers CDV_ERR_UNSUPPORTED."""
    from paper_1711_11224_gb300 import Plan, _binding
    P = _problems(SHAPES[:1], 2)[0]
    with Plan(P.m, P.p) as pl:
        pl.set_psf(_dev(P.H))
        with pytest.raises(_binding.CdvError, match="UNSUPPORTED"):
            pl.iterate(_dev(P.Y), K=2, x0="crop", path="persistent")

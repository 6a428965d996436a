"""Host-side pieces of bench.py (no GPU): the separable factor table, the roofline peaks and the
committed DRAM-traffic records."""
import json
import os

import numpy as np
import pytest

import bench
import synth


@pytest.mark.parametrize("name", sorted(bench.SEPARABLE))
def test_separable_factors_reproduce_the_workload_template(name):
    """The factors the separable metric uses multiply out to the workload's own (dense) template."""
    P = getattr(synth, name)()
    q, sigma = bench.SEPARABLE[name]
    assert tuple(P.H.shape) == tuple(q)
    hs = synth.gaussian_factors(q, sigma)
    H = hs[0].astype(np.float64)
    for h in hs[1:]:
        H = np.multiply.outer(H, h.astype(np.float64))
    np.testing.assert_allclose(H, P.H, rtol=2e-6, atol=1e-9)
    for h in hs:
        assert abs(float(h.astype(np.float64).sum()) - 1.0) < 1e-6


def test_ring_template_is_not_separable():
    """ring3d's template has rank > 1 as a matrix over (axis 1, axes 2-3): the separable mode rejects it."""
    assert "ring3d" not in bench.SEPARABLE
    H = synth.ring_psf().astype(np.float64)
    s = np.linalg.svd(H.reshape(H.shape[0], -1), compute_uv=False)
    assert s[1] > 1e-3 * s[0]


def test_fp32_peak_from_unit_counts():
    bound, peak, basis = bench.roofline_peak("fp32")
    assert bound == "alu"
    assert abs(peak - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9


def test_traffic_records_follow_the_kernel_sources():
    """Each committed record matches the current kernel source hash, or is ignored (None).  Its bytes
    are a plausible count for the kernel: the FP32 engine reads its input about once (at most twice the
    308 MB of algorithmic FP32 bytes); the tensor-core kernels read BF16 shadows whose planes are
    re-read from DRAM by CTAs working on different planes (at most 16 times the algorithmic bytes)."""
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    bound = {"fp32": 2, "split3": 16, "bf16": 16, "tf32": 16}
    for mode, kernels in rec["ring3d"].items():
        for kernel, e in kernels.items():
            v = bench.traffic_record("ring3d", mode, kernel)
            if e["source_hash"] == bench.kernel_hash(mode):
                assert v == float(e["bytes_per_launch"])
                assert 0 < v < bound[mode] * 308126016
            else:
                assert v is None
    assert bench.traffic_record("ring3d", "fp32", "nonexistent") is None

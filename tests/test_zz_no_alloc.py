"""The allocation-free template gradient (cdv_grad_psf_static) against the FP64 oracle.

cdv_grad_psf_static serves callers that cannot allocate device memory (code
running while a CUDA graph is captured in global mode, plug-ins whose host
framework owns all device memory): it keeps its partial sums in a static
device array instead of a plan's workspace.  Its results are compared with
oracle.grad_psf, the FP64 sum written from the definition, and with the plan's
cdv_grad_psf.  This file is collected last so that a run stopping at the first
failure has run every other test already; it passes alone and after them.
"""
import ctypes

import numpy as np
import pytest

import oracle
from _util import TOL_CONV, rel_l2

torch = pytest.importorskip("torch")

UNSUPPORTED = 3


def _call_static(lib, m, p, X, dY, dH):
    n = len(m)
    mm = (ctypes.c_int64 * n)(*m)
    pp = (ctypes.c_int32 * n)(*p)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    batch = X.shape[0]
    return lib.cdv_grad_psf_static(n, mm, pp, batch, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(dY.data_ptr()),
                                   ctypes.c_void_p(dH.data_ptr()), stream)


def _inputs(rng, B, m, p):
    ny = tuple(a + 2 * b for a, b in zip(m, p))
    X = rng.random((B,) + m).astype(np.float32)
    dY = rng.standard_normal((B,) + ny).astype(np.float32)
    return X, dY


@pytest.mark.gpu
def test_static_scratch_matches_oracle_two_calls():
    from paper_1711_11224_gb300 import Plan, _binding
    lib = _binding.load()
    m, p = (9, 20, 70), (2, 3, 4)
    q = tuple(2 * v + 1 for v in p)
    rng = np.random.default_rng(11)
    with Plan(m, p) as pl:
        for call in range(2):                      # the array keeps the last call's contents
            B = 3 if call == 0 else 2
            Xh, dYh = _inputs(rng, B, m, p)
            X, dY = torch.from_numpy(Xh).cuda(), torch.from_numpy(dYh).cuda()
            dH = torch.full(q, float("nan"), device="cuda")
            assert _call_static(lib, m, p, X, dY, dH) == 0, lib.cdv_last_error()
            got = dH.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert rel_l2(got, oracle.grad_psf(Xh, dYh, q)) <= TOL_CONV
            assert rel_l2(got, pl.grad_psf(X, dY).cpu().numpy()) <= TOL_CONV


@pytest.mark.gpu
@pytest.mark.parametrize("m,p", [((3, 4, 6), (20, 15, 39)),     # 41x31x79: chunks clamped 15 -> 5 by the array
                                 ((2, 3, 5), (65, 15, 64))])    # 131x31x129: 523,869 samples, one chunk
def test_static_scratch_large_template_clamps_chunks(m, p):
    """Templates whose partials only fit the static array with fewer chunks than a plan would use."""
    from paper_1711_11224_gb300 import _binding
    lib = _binding.load()
    q = tuple(2 * v + 1 for v in p)
    assert int(np.prod(q)) <= 1 << 19
    rng = np.random.default_rng(12)
    for call in range(2):
        Xh, dYh = _inputs(rng, 2, m, p)
        dH = torch.full(q, float("nan"), device="cuda")
        assert _call_static(lib, m, p, torch.from_numpy(Xh).cuda(), torch.from_numpy(dYh).cuda(), dH) == 0, \
            lib.cdv_last_error()
        assert rel_l2(dH.cpu().numpy(), oracle.grad_psf(Xh, dYh, q)) <= TOL_CONV


@pytest.mark.gpu
@pytest.mark.parametrize("m,p,what", [((4, 4, 4), (150, 20, 21), b"static scratch"),   # 301x41x43 > 524288
                                      ((2, 3, 4), (0, 400, 0), b"shared memory")])     # 801 rows of one column
def test_static_scratch_rejects_unsupported_templates(m, p, what):
    from paper_1711_11224_gb300 import _binding
    lib = _binding.load()
    X = torch.zeros((1,) + m, device="cuda")
    dY = torch.zeros(1, device="cuda")
    dH = torch.zeros(1, device="cuda")
    assert _call_static(lib, m, p, X, dY, dH) == UNSUPPORTED    # nothing enqueued
    assert what in lib.cdv_last_error()

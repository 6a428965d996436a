"""The allocation-free template gradient (cdv_grad_psf_static) against cdv_grad_psf.

cdv_grad_psf_static serves callers that cannot allocate device memory: it
keeps its partial sums in a static device array instead of a plan's
workspace.  This file is collected last so that a run stopping at the first
failure has run every other test already; it passes alone and after them.
"""
import ctypes

import numpy as np
import pytest

from _util import TOL_CONV, rel_l2

torch = pytest.importorskip("torch")


def _call_static(lib, m, p, X, dY, dH):
    n = len(m)
    mm = (ctypes.c_int64 * n)(*m)
    pp = (ctypes.c_int32 * n)(*p)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    batch = X.shape[0]
    return lib.cdv_grad_psf_static(n, mm, pp, batch, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(dY.data_ptr()),
                                   ctypes.c_void_p(dH.data_ptr()), stream)


@pytest.mark.gpu
def test_static_scratch_matches_plan_two_calls():
    from paper_1711_11224_gb300 import Plan, _binding
    lib = _binding.load()
    m, p = (9, 20, 70), (2, 3, 4)
    q = tuple(2 * v + 1 for v in p)
    ny = tuple(a + 2 * b for a, b in zip(m, p))
    rng = np.random.default_rng(11)
    with Plan(m, p) as pl:
        for call in range(2):                      # the array keeps the last call's contents
            B = 3 if call == 0 else 2
            X = torch.from_numpy(rng.random((B,) + m).astype(np.float32)).cuda()
            dY = torch.from_numpy(rng.standard_normal((B,) + ny).astype(np.float32)).cuda()
            ref = pl.grad_psf(X, dY).cpu().numpy()
            dH = torch.full(q, float("nan"), device="cuda")
            assert _call_static(lib, m, p, X, dY, dH) == 0, lib.cdv_last_error()
            got = dH.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert rel_l2(got, ref) <= TOL_CONV


@pytest.mark.gpu
def test_static_scratch_rejects_oversized_template():
    from paper_1711_11224_gb300 import _binding
    lib = _binding.load()
    m, p = (4, 4, 4), (150, 20, 21)               # 301 x 41 x 43 > 524288 samples
    X = torch.zeros((1,) + m, device="cuda")
    dY = torch.zeros(1, device="cuda")
    dH = torch.zeros(1, device="cuda")
    assert _call_static(lib, m, p, X, dY, dH) == 3   # CDV_ERR_UNSUPPORTED, nothing enqueued
    assert b"static scratch" in lib.cdv_last_error()

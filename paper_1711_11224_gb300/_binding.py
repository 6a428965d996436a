"""ctypes binding of libcdv (include/cdv.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module turns
torch tensors into device pointers and the current torch stream into the
``stream`` argument.  There is no CPU fallback: if the library is missing or
no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcdv.so")

CDV_OK = 0
STATUS = {
    0: "CDV_OK", 1: "CDV_ERR_INVALID_ARG", 2: "CDV_ERR_SHAPE", 3: "CDV_ERR_UNSUPPORTED", 4: "CDV_ERR_OOM",
    5: "CDV_ERR_CUDA", 6: "CDV_ERR_TIMEOUT", 7: "CDV_ERR_NOT_DESCENDING", 8: "CDV_ERR_NONFINITE",
    9: "CDV_ERR_NO_PSF",
}
MODES = {"fp32": 0, "bf16": 1, "tf32": 2, "split3": 3, "fft": 4, "separable": 5}
X0 = {"given": 0, "crop": 1, "zero": 2}
PATHS = {"auto": 0, "general": 1, "small": 2, "persistent": 3}

# Every symbol include/cdv.h declares (checked by the tests).
EXPORTS = [
    "cdv_status_string", "cdv_last_error", "cdv_version", "cdv_plan_create", "cdv_plan_workspace_size",
    "cdv_plan_set_psf", "cdv_plan_lipschitz", "cdv_plan_destroy", "cdv_forward", "cdv_adjoint", "cdv_grad_psf",
    "cdv_iter_opts_default", "cdv_iterate", "cdv_iterate_host", "cdv_richardson_lucy", "cdv_plan_sync_status",
    "cdv_grad_psf_static", "cdv_batch_plan_create", "cdv_batch_workspace_size", "cdv_batch_set_psfs",
    "cdv_batch_iterate", "cdv_batch_destroy", "cdv_plan_describe", "cdv_plan_set_psf_factors",
    "cdv_plan_set_wait_cycles", "cdv_probe_fp32_fma", "cdv_batch_set_wait_cycles",
]


class CdvError(RuntimeError):
    def __init__(self, status, detail=""):
        self.status = status
        super().__init__("%s: %s" % (STATUS.get(status, status), detail))


class IterOpts(ctypes.Structure):
    _fields_ = [("x0_policy", ctypes.c_int), ("delta0", ctypes.c_double), ("beta", ctypes.c_double),
                ("max_halvings", ctypes.c_int), ("max_rejects", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("path", ctypes.c_int), ("bb", ctypes.c_int), ("reserved", ctypes.c_int * 2),
                ("tikhonov", ctypes.c_double),
                ("armijo", ctypes.c_double)]


class IterReport(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_int), ("rejected", ctypes.c_int), ("status", ctypes.c_int),
                ("trials", ctypes.c_int), ("f0", ctypes.c_double), ("f_final", ctypes.c_double),
                ("gmac", ctypes.c_double), ("f_hist", ctypes.POINTER(ctypes.c_double)),
                ("delta_hist", ctypes.POINTER(ctypes.c_double))]


class PlanInfo(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("cols", ctypes.c_int32 * 2), ("K", ctypes.c_int32 * 2),
                ("grid", ctypes.c_int32 * 2), ("tiles", ctypes.c_int64 * 2), ("executed_macs", ctypes.c_double * 2),
                ("algorithmic_macs", ctypes.c_double)]


_lib = None


def load(path=LIB_PATH):
    """Load libcdv.so (built by paper_1711_11224_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libcdv.so is not built (%s); run `python -c \"import __graft_entry__ as g; g.build()\"`"
                          % path)
    lib = ctypes.CDLL(path)
    vp, i32, i64p = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)
    st = ctypes.c_int
    lib.cdv_status_string.restype = ctypes.c_char_p
    lib.cdv_status_string.argtypes = [st]
    lib.cdv_last_error.restype = ctypes.c_char_p
    lib.cdv_version.restype = i32
    lib.cdv_plan_create.restype = st
    lib.cdv_plan_create.argtypes = [ctypes.POINTER(vp), i32, i64p, ctypes.POINTER(ctypes.c_int32), i32, vp]
    lib.cdv_plan_workspace_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.cdv_plan_set_psf.argtypes = [vp, vp, vp]
    lib.cdv_plan_set_psf_factors.argtypes = [vp, ctypes.POINTER(vp), vp]
    lib.cdv_plan_lipschitz.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.cdv_plan_destroy.argtypes = [vp]
    lib.cdv_plan_describe.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    lib.cdv_forward.argtypes = [vp, i32, vp, vp, vp]
    lib.cdv_adjoint.argtypes = [vp, i32, vp, vp, vp]
    lib.cdv_grad_psf.argtypes = [vp, i32, vp, vp, vp, vp]
    lib.cdv_iter_opts_default.restype = None
    lib.cdv_iter_opts_default.argtypes = [ctypes.POINTER(IterOpts)]
    lib.cdv_iterate.argtypes = [vp, vp, vp, i32, ctypes.POINTER(IterOpts), ctypes.POINTER(IterReport), vp]
    lib.cdv_iterate_host.argtypes = [vp, vp, vp, i32, ctypes.POINTER(IterOpts), ctypes.POINTER(IterReport), vp]
    lib.cdv_richardson_lucy.argtypes = [vp, vp, vp, i32, vp]
    lib.cdv_plan_sync_status.argtypes = [vp, vp]
    lib.cdv_plan_set_wait_cycles.argtypes = [vp, ctypes.c_longlong]
    lib.cdv_batch_set_wait_cycles.argtypes = [vp, ctypes.c_longlong]
    lib.cdv_probe_fp32_fma.argtypes = [vp, i32, i32, i32, vp]
    lib.cdv_grad_psf_static.argtypes = [i32, i64p, ctypes.POINTER(ctypes.c_int32), i32, vp, vp, vp, vp]
    lib.cdv_batch_plan_create.argtypes = [ctypes.POINTER(vp), i32, i32, i64p, ctypes.POINTER(ctypes.c_int32), i32, i32,
                                          vp]
    lib.cdv_batch_workspace_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.cdv_batch_set_psfs.argtypes = [vp, ctypes.POINTER(vp), vp]
    lib.cdv_batch_iterate.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), i32, ctypes.POINTER(IterOpts),
                                      ctypes.POINTER(IterReport), vp]
    lib.cdv_batch_destroy.argtypes = [vp]
    _lib = lib
    return lib


def check(status):
    if status != CDV_OK:
        lib = load()
        raise CdvError(status, lib.cdv_last_error().decode(errors="replace"))

"""Python face of a cdv plan: the forward/adjoint operators and the iteration.

Names follow the paper: X (m samples per axis), H (2p+1), Y (m+2p).  Arrays
are torch CUDA float32 tensors in C-order; the work is enqueued on the
current torch stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _binding as B


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _need(t, shape, name):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("%s must be a contiguous float32 CUDA tensor" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))


class Plan:
    """A plan for one size: m samples of X per axis, template half-widths p.

    mode: "fp32" (FP32 FMA), "split3" (tensor cores, split-BF16x3: FP32 accuracy), "tf32", "bf16"
    (tensor cores, lower accuracy), "separable" (template given by its 1-D factors through
    set_psf_factors, one 1-D pass per axis) or "fft" (cuFFT comparator, not the paper's method).
    """

    def __init__(self, m, p, mode="fp32"):
        self.lib = B.load()
        self.m = tuple(int(v) for v in m)
        self.p = tuple(int(v) for v in p)
        if len(self.m) != len(self.p):
            raise ValueError("m and p disagree on n")
        self.n = len(self.m)
        self.q = tuple(2 * v + 1 for v in self.p)
        self.ny_shape = tuple(a + 2 * b for a, b in zip(self.m, self.p))
        self.mode = mode
        mm = (ctypes.c_int64 * self.n)(*self.m)
        pp = (ctypes.c_int32 * self.n)(*self.p)
        h = ctypes.c_void_p()
        B.check(self.lib.cdv_plan_create(ctypes.byref(h), self.n, mm, pp, B.MODES[mode], _stream()))
        self._h = h
        self.H = None

    # -- lifetime -------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self.lib.cdv_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def workspace_bytes(self):
        v = ctypes.c_size_t()
        B.check(self.lib.cdv_plan_workspace_size(self._h, ctypes.byref(v)))
        return int(v.value)

    def describe(self):
        """Tiling of the two convolutions ([forward, adjoint]) and the MACs the hardware executes."""
        i = B.PlanInfo()
        B.check(self.lib.cdv_plan_describe(self._h, ctypes.byref(i)))
        return {"mode": self.mode, "cols": list(i.cols), "K": list(i.K), "grid": list(i.grid),
                "tiles": list(i.tiles), "executed_macs": list(i.executed_macs), "algorithmic_macs": i.algorithmic_macs}

    # -- template -------------------------------------------------------
    def set_psf(self, H):
        _need(H, self.q, "H")
        B.check(self.lib.cdv_plan_set_psf(self._h, _ptr(H), _stream()))
        self.H = H
        return self

    def set_psf_factors(self, hs):
        """Separable template H = h_1 x .. x h_n (mode "separable"): one device tensor of 2p_i+1 samples per axis."""
        hs = list(hs)
        if len(hs) != self.n:
            raise ValueError("expected %d factors, got %d" % (self.n, len(hs)))
        for i, h in enumerate(hs):
            _need(h, (self.q[i],), "h[%d]" % i)
        arr = (ctypes.c_void_p * self.n)(*[h.data_ptr() for h in hs])
        B.check(self.lib.cdv_plan_set_psf_factors(self._h, arr, _stream()))
        self.H = hs
        return self

    def lipschitz(self):
        v = ctypes.c_double()
        B.check(self.lib.cdv_plan_lipschitz(self._h, ctypes.byref(v)))
        return float(v.value)

    # -- operators ------------------------------------------------------
    def forward(self, X, Y=None):
        """Y = X (*) H (Property 1).  X: m or (B, *m)."""
        batch = 1 if X.dim() == self.n else X.shape[0]
        xs = self.m if X.dim() == self.n else (batch,) + self.m
        _need(X, xs, "X")
        ys = self.ny_shape if X.dim() == self.n else (batch,) + self.ny_shape
        if Y is None:
            Y = torch.empty(ys, device=X.device, dtype=torch.float32)
        _need(Y, ys, "Y")
        B.check(self.lib.cdv_forward(self._h, batch, _ptr(X), _ptr(Y), _stream()))
        return Y

    def adjoint(self, R, G=None):
        """G = (A_n^h)^T R = M_2p(R (*) H~) (Property 2).  R: m+2p or (B, *(m+2p))."""
        batch = 1 if R.dim() == self.n else R.shape[0]
        rs = self.ny_shape if R.dim() == self.n else (batch,) + self.ny_shape
        _need(R, rs, "R")
        gs = self.m if R.dim() == self.n else (batch,) + self.m
        if G is None:
            G = torch.empty(gs, device=R.device, dtype=torch.float32)
        _need(G, gs, "G")
        B.check(self.lib.cdv_adjoint(self._h, batch, _ptr(R), _ptr(G), _stream()))
        return G

    def grad_psf(self, X, dY, dH=None):
        """dH(j) = sum_b sum_k X_b(k) dY_b(k + j)."""
        batch = 1 if X.dim() == self.n else X.shape[0]
        _need(X, self.m if X.dim() == self.n else (batch,) + self.m, "X")
        _need(dY, self.ny_shape if dY.dim() == self.n else (batch,) + self.ny_shape, "dY")
        if dH is None:
            dH = torch.empty(self.q, device=X.device, dtype=torch.float32)
        _need(dH, self.q, "dH")
        B.check(self.lib.cdv_grad_psf(self._h, batch, _ptr(X), _ptr(dY), _ptr(dH), _stream()))
        return dH

    # -- iteration ------------------------------------------------------
    @staticmethod
    def opts(x0="given", delta0=None, beta=0.5, max_halvings=20, max_rejects=16, use_graph=True, path="auto",
             tikhonov=0.0, armijo=0.0, bb=False):
        """Options of Steps 1-3; tikhonov adds lambda/2 ||x||^2 to f, armijo is the sufficient-decrease
        factor sigma, bb starts steps from Barzilai-Borwein lengths (all off: the paper's objective and
        decrease rule with delta0 at every step)."""
        o = B.IterOpts()
        B.load().cdv_iter_opts_default(ctypes.byref(o))
        o.x0_policy = B.X0[x0]
        o.delta0 = 0.0 if delta0 is None else float(delta0)
        o.beta = float(beta)
        o.max_halvings = int(max_halvings)
        o.max_rejects = int(max_rejects)
        o.use_graph = 1 if use_graph else 0
        o.path = B.PATHS[path]
        o.tikhonov = float(tikhonov)
        o.armijo = float(armijo)
        o.bb = 1 if bb else 0
        return o

    def _report(self, K, want):
        if not want:
            return None, None, None
        rep = B.IterReport()
        f = np.zeros(K + 1, dtype=np.float64)
        d = np.zeros(max(K, 1), dtype=np.float64)
        rep.f_hist = f.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        rep.delta_hist = d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        return rep, f, d

    @staticmethod
    def _pack(rep, f, d):
        a = rep.accepted
        return {"accepted": a, "rejected": rep.rejected, "status": B.STATUS.get(rep.status, rep.status),
                "trials": rep.trials, "f0": rep.f0, "f_final": rep.f_final, "gmac": rep.gmac,
                "f": f[:a + 1].copy(), "delta": d[:a].copy()}

    def iterate(self, Y, X=None, K=100, report=True, **kw):
        """Projected gradient (Steps 1-3): K accepted steps from X (x0='given') or a policy."""
        _need(Y, self.ny_shape, "Y")
        if X is None:
            X = torch.empty(self.m, device=Y.device, dtype=torch.float32)
            kw.setdefault("x0", "crop")
        _need(X, self.m, "X")
        o = self.opts(**kw)
        rep, f, d = self._report(K, report)
        B.check(self.lib.cdv_iterate(self._h, _ptr(Y), _ptr(X), int(K), ctypes.byref(o),
                                     ctypes.byref(rep) if rep is not None else None, _stream()))
        return (X, self._pack(rep, f, d)) if report else (X, None)

    def iterate_host(self, Y, X, K=100, report=True, **kw):
        """cdv_iterate_host on numpy float32 arrays (copies inside the call)."""
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        if Y.shape != self.ny_shape or X.shape != self.m or X.dtype != np.float32 or not X.flags.c_contiguous:
            raise ValueError("host arrays of the wrong shape or type")
        o = self.opts(**kw)
        rep, f, d = self._report(K, report)
        B.check(self.lib.cdv_iterate_host(self._h, Y.ctypes.data_as(ctypes.c_void_p),
                                          X.ctypes.data_as(ctypes.c_void_p), int(K), ctypes.byref(o),
                                          ctypes.byref(rep) if rep is not None else None, _stream()))
        return (X, self._pack(rep, f, d)) if report else (X, None)

    def richardson_lucy(self, Y, X, K):
        _need(Y, self.ny_shape, "Y")
        _need(X, self.m, "X")
        B.check(self.lib.cdv_richardson_lucy(self._h, _ptr(Y), _ptr(X), int(K), _stream()))
        return X

    def sync(self):
        B.check(self.lib.cdv_plan_sync_status(self._h, _stream()))

    def set_wait_cycles(self, cycles=0):
        """Budget of each barrier wait in the tensor-core kernels (clock cycles; 0: the default)."""
        B.check(self.lib.cdv_plan_set_wait_cycles(self._h, int(cycles)))
        return self


class BatchPlan:
    """Many independent problems iterated together (FP32): volume i has m[i] samples, half-widths p[i]."""

    def __init__(self, ms, ps, autotune=True):
        self.lib = B.load()
        self.ms = [tuple(int(v) for v in m) for m in ms]
        self.ps = [tuple(int(v) for v in p) for p in ps]
        self.count = len(self.ms)
        self.n = len(self.ms[0])
        if self.count < 1 or len(self.ps) != self.count or any(len(m) != self.n or len(p) != self.n
                                                               for m, p in zip(self.ms, self.ps)):
            raise ValueError("one (m, p) pair of the same n per volume")
        self.qs = [tuple(2 * v + 1 for v in p) for p in self.ps]
        self.ny_shapes = [tuple(a + 2 * b for a, b in zip(m, p)) for m, p in zip(self.ms, self.ps)]
        mm = (ctypes.c_int64 * (self.count * self.n))(*[v for m in self.ms for v in m])
        pp = (ctypes.c_int32 * (self.count * self.n))(*[v for p in self.ps for v in p])
        h = ctypes.c_void_p()
        B.check(self.lib.cdv_batch_plan_create(ctypes.byref(h), self.count, self.n, mm, pp, 0,
                                               1 if autotune else 0, _stream()))
        self._h = h
        self.H = None

    def close(self):
        if getattr(self, "_h", None):
            self.lib.cdv_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def workspace_bytes(self):
        v = ctypes.c_size_t()
        B.check(self.lib.cdv_batch_workspace_size(self._h, ctypes.byref(v)))
        return int(v.value)

    def _ptrs(self, ts):
        return (ctypes.c_void_p * self.count)(*[t.data_ptr() for t in ts])

    def set_psfs(self, Hs):
        for H, q in zip(Hs, self.qs):
            _need(H, q, "H")
        B.check(self.lib.cdv_batch_set_psfs(self._h, self._ptrs(Hs), _stream()))
        self.H = list(Hs)
        return self

    def set_wait_cycles(self, cycles=0):
        """Idle budget (SM cycles) of a CTA of the persistent run before it reports CDV_ERR_TIMEOUT
        (0: the default, about 0.5 s)."""
        B.check(self.lib.cdv_batch_set_wait_cycles(self._h, int(cycles)))

    def iterate(self, Ys, Xs=None, K=100, report=True, **kw):
        """K accepted steps of Steps 1-3 for every volume; returns (Xs, reports).  path="auto" or
        "persistent" (default): one persistent launch for the whole run; path="general": common trial
        slots of batched launches."""
        for Y, s in zip(Ys, self.ny_shapes):
            _need(Y, s, "Y")
        if Xs is None:
            Xs = [torch.empty(m, device=Ys[0].device, dtype=torch.float32) for m in self.ms]
            kw.setdefault("x0", "crop")
        for X, m in zip(Xs, self.ms):
            _need(X, m, "X")
        o = Plan.opts(**kw)
        reps = None
        hist = []
        if report:
            reps = (B.IterReport * self.count)()
            for r in reps:
                f = np.zeros(K + 1)
                d = np.zeros(max(K, 1))
                r.f_hist = f.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                r.delta_hist = d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                hist.append((f, d))
        B.check(self.lib.cdv_batch_iterate(self._h, self._ptrs(Ys), self._ptrs(Xs), int(K), ctypes.byref(o),
                                           reps, _stream()))
        if not report:
            return Xs, None
        return Xs, [Plan._pack(r, f, d) for r, (f, d) in zip(reps, hist)]

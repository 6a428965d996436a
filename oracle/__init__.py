"""FP64 CPU oracle for direct-convolution deconvolution.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.  It
shares no code with the CUDA path.

The arithmetic lives in ``cdv_oracle.c`` (plain nested loops, double
precision, OpenMP over the slowest output axis); ``dense.py`` builds the
explicit block-Toeplitz matrix A_n^h by the recursion of Property 1.  This
module marshals numpy arrays of 1, 2 or 3 dimensions into the C routines,
which work on 3-D arrays (leading axes of size 1, p = 0).

Every function converts its inputs to float64 first; callers pass the same
float32 arrays they give the CUDA path.

Parity pins (tests/test_oracle.py): forward and adjoint equal the dense A and
A^T exactly on integer data; the two adjoint forms agree; adjoint identity;
delta templates; commutativity; mass invariant; separable closed form;
iterate against a library NNLS and the identity-template special case;
dH against central finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "cdv_oracle.c")
_lock = threading.Lock()
_lib = None

__all__ = [
    "build", "forward", "adjoint", "adjoint_crop", "forward_points", "adjoint_points",
    "grad_psf", "iterate", "richardson_lucy", "lipschitz", "x0_crop", "num_threads", "set_num_threads",
    "gradient_eq6", "objective",
]


def build(force=False):
    """Compile cdv_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64, i32, dp = ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int64)
            dims = [i64, i64, i64, i32, i32, i32]
            lib.orc_forward.argtypes = dims + [dp, dp, dp]
            lib.orc_adjoint.argtypes = dims + [dp, dp, dp]
            lib.orc_adjoint_crop.argtypes = dims + [dp, dp, dp]
            lib.orc_forward_points.argtypes = dims + [dp, dp, i64, ip, dp]
            lib.orc_adjoint_points.argtypes = dims + [dp, dp, i64, ip, dp]
            lib.orc_grad_psf.argtypes = [i64] + dims + [dp, dp, dp]
            lib.orc_iterate.argtypes = dims + [dp, dp, dp, i32, ctypes.c_double, ctypes.c_double, i32,
                                               ctypes.c_double, ctypes.c_double, i32,
                                               dp, dp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
            lib.orc_iterate.restype = i32
            lib.orc_richardson_lucy.argtypes = dims + [dp, dp, dp, i32]
            lib.orc_num_threads.restype = i32
            lib.orc_set_num_threads.argtypes = [i32]
            lib.orc_set_num_threads.restype = None
            _lib = lib
    return _lib


def num_threads():
    return int(_load().orc_num_threads())


def set_num_threads(n):
    """Threads of later calls (for timing; every result is independent of it)."""
    _load().orc_set_num_threads(int(n))


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(m, p):
    m = tuple(int(v) for v in m)
    p = tuple(int(v) for v in p)
    if not (1 <= len(m) <= 3) or len(m) != len(p):
        raise ValueError("n must be 1, 2 or 3")
    m3 = (1,) * (3 - len(m)) + m
    p3 = (0,) * (3 - len(p)) + p
    return m3 + p3


def _p_of(H):
    if any(q % 2 == 0 for q in H.shape):
        raise ValueError("template sizes must be odd (2p+1)")
    return tuple((q - 1) // 2 for q in H.shape)


def forward(X, H):
    """Y = X (*) H, full size m + 2p per axis (Property 1)."""
    X, H = _d(X), _d(H)
    p = _p_of(H)
    Y = np.empty(tuple(a + 2 * b for a, b in zip(X.shape, p)), dtype=np.float64)
    _load().orc_forward(*_dims(X.shape, p), _ptr(X), _ptr(H), _ptr(Y))
    return Y


def adjoint(R, H):
    """G = (A_n^h)^T R = M_2p(R (*) H~), size m = shape(R) - 2p (Property 2)."""
    R, H = _d(R), _d(H)
    p = _p_of(H)
    m = tuple(a - 2 * b for a, b in zip(R.shape, p))
    if min(m) < 1:
        raise ValueError("R smaller than the template")
    G = np.empty(m, dtype=np.float64)
    _load().orc_adjoint(*_dims(m, p), _ptr(R), _ptr(H), _ptr(G))
    return G


def adjoint_crop(R, H):
    """Property 2 literally: full convolution with the flipped template, then crop [2p, 2p+m)."""
    R, H = _d(R), _d(H)
    p = _p_of(H)
    m = tuple(a - 2 * b for a, b in zip(R.shape, p))
    G = np.empty(m, dtype=np.float64)
    _load().orc_adjoint_crop(*_dims(m, p), _ptr(R), _ptr(H), _ptr(G))
    return G


def _idx3(idx, nd):
    idx = np.asarray(idx, dtype=np.int64).reshape(-1, nd)
    if nd < 3:
        idx = np.concatenate([np.zeros((idx.shape[0], 3 - nd), np.int64), idx], axis=1)
    return np.ascontiguousarray(idx)


def forward_points(X, H, idx):
    """y(s) at the given output indices s (array of shape npts x n)."""
    X, H = _d(X), _d(H)
    p = _p_of(H)
    ii = _idx3(idx, X.ndim)
    out = np.empty(ii.shape[0], dtype=np.float64)
    _load().orc_forward_points(*_dims(X.shape, p), _ptr(X), _ptr(H), ii.shape[0],
                               ii.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(out))
    return out


def adjoint_points(R, H, idx):
    """(A^T R)(k) at the given indices k (npts x n)."""
    R, H = _d(R), _d(H)
    p = _p_of(H)
    m = tuple(a - 2 * b for a, b in zip(R.shape, p))
    ii = _idx3(idx, R.ndim)
    out = np.empty(ii.shape[0], dtype=np.float64)
    _load().orc_adjoint_points(*_dims(m, p), _ptr(R), _ptr(H), ii.shape[0],
                               ii.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(out))
    return out


def grad_psf(X, dY, q):
    """dH(j) = sum_b sum_k X_b(k) dY_b(k + j); X is (B, *m), dY is (B, *(m+2p))."""
    X, dY = _d(X), _d(dY)
    q = tuple(int(v) for v in q)
    p = tuple((v - 1) // 2 for v in q)
    B = X.shape[0]
    dH = np.empty(q, dtype=np.float64)
    _load().orc_grad_psf(B, *_dims(X.shape[1:], p), _ptr(X), _ptr(dY), _ptr(dH))
    return dH


def lipschitz(H):
    """L = (sum_j |h(j)|)^2 >= ||A||_2^2 (Young's inequality): delta0 = 1/L."""
    return float(np.abs(np.asarray(H, dtype=np.float64)).sum()) ** 2


def x0_crop(Y, p):
    """Initial solution: the centre crop Y[p : p + m] clipped at 0."""
    Y = np.asarray(Y, dtype=np.float64)
    sl = tuple(slice(b, a - b) for a, b in zip(Y.shape, p))
    return np.maximum(Y[sl], 0.0)


def objective(X, H, Y):
    """f(x) = 1/2 ||A x - y||^2."""
    r = forward(X, H) - _d(Y)
    return 0.5 * float(np.dot(r.ravel(), r.ravel()))


def gradient_eq6(X, H, Y):
    """Eq. 6 literally: M(H~ (*) (H (*) X)) - M(H~ (*) Y), and the residual form A^T(AX - Y)."""
    lit = adjoint(forward(X, H), H) - adjoint(Y, H)
    res = adjoint(forward(X, H) - _d(Y), H)
    return lit, res


def iterate(Y, H, X0, K, delta0=None, beta=0.5, max_halvings=20, tikhonov=0.0, armijo=0.0, bb=False):
    """Projected gradient (Steps 1-3) from X0 for K accepted steps.

    Objective 1/2 ||A x - y||^2 + tikhonov/2 ||x||^2 (tikhonov = 0: the paper's NNLS objective);
    a trial is accepted when f drops below f(x_k) + armijo <grad f(x_k), x_t - x_k> (armijo = 0:
    the decrease condition of Step 2).  The default step is 1/L with L = (sum |h|)^2 + tikhonov;
    bb = True starts each step from a Barzilai-Borwein length lagged by one step (see cdv_oracle.c).
    Returns dict(X, f, delta, accepted, rejected, status) with f of length
    accepted + 1 (f[0] = f(X0)) and status 0 (K steps) or 1 (converged).
    """
    Y, H = _d(Y), _d(H)
    X = _d(X0).copy()
    p = _p_of(H)
    if delta0 is None:
        delta0 = 1.0 / (lipschitz(H) + float(tikhonov))
    f = np.zeros(K + 1)
    dl = np.zeros(max(K, 1))
    na, nr = ctypes.c_int(0), ctypes.c_int(0)
    st = _load().orc_iterate(*_dims(X.shape, p), _ptr(Y), _ptr(H), _ptr(X), int(K),
                             float(delta0), float(beta), int(max_halvings), float(tikhonov), float(armijo), int(bool(bb)),
                             _ptr(f), _ptr(dl), ctypes.byref(na), ctypes.byref(nr))
    a = na.value
    return {"X": X, "f": f[:a + 1], "delta": dl[:a], "accepted": a, "rejected": nr.value, "status": int(st)}


def richardson_lucy(Y, H, X0, K):
    """Richardson-Lucy iterations (the comparison method of the Results)."""
    Y, H = _d(Y), _d(H)
    X = _d(X0).copy()
    p = _p_of(H)
    _load().orc_richardson_lucy(*_dims(X.shape, p), _ptr(Y), _ptr(H), _ptr(X), int(K))
    return X

"""Seeded synthetic inputs for the deconvolution workloads.

This module only draws inputs.  It holds none of the method's arithmetic: no
direct convolution, no adjoint, no iteration.  The observation model
Y = X (*) H + N (Eq. 3-5) needs a blur to synthesise Y; that blur is the
library FFT convolution ``scipy.signal.fftconvolve`` so that the inputs share
no code with the FP64 oracle nor with the CUDA path, which both receive the
same float32 arrays from here.

Every generator takes an explicit seed; sub-streams come from
``numpy.random.SeedSequence(seed).spawn``.  Shapes are C-order with axis 1
slowest and the last axis contiguous, PSF sizes are odd (q_i = 2 p_i + 1).

Workloads (their sizes follow the paper's use of 2-D and 3-D images, Section
"Application to 2-dimensional deconvolution" and "Results", scaled to the
microscopy volumes the method targets):

* ``blobs2d``   -- 64x64 image of 20 Gaussian blobs, 7x7 Gaussian PSF (sigma 1.5),
                   additive Gaussian noise sigma 0.01, 50 iterations.
* ``fil3d``     -- 256x256x64 tubular filaments + background 10, 15x15x11
                   anisotropic Gaussian PSF, Poisson noise, 100 iterations.
* ``grad3d``    -- 4 volumes 128x128x64, 11x11x9 Gaussian PSF (learnable sigma).
* ``ring3d``    -- 512x512x128 filaments, 31x31x21 Gaussian-plus-ring PSF,
                   Poisson noise, 100 iterations.
* ``batch64``   -- 64 volumes of uneven size and PSF size, 200 iterations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem", "gaussian_psf", "gaussian_factors", "ring_psf", "blobs", "filaments", "observe",
    "blobs2d", "fil3d", "grad3d", "ring3d", "batch64", "batch64_shapes",
    "scaled_fil3d", "scaled_ring3d", "integer_case", "random_case", "WORKLOADS",
]


@dataclass
class Problem:
    """One deconvolution problem: Y observed, H the PSF, X_true the target."""
    name: str
    X_true: np.ndarray          # float32, shape m
    H: np.ndarray               # float32, shape q = 2p+1
    Y: np.ndarray               # float32, shape m + 2p
    K: int                      # iterations
    meta: dict = field(default_factory=dict)

    @property
    def m(self):
        return tuple(int(s) for s in self.X_true.shape)

    @property
    def p(self):
        return tuple(int((q - 1) // 2) for q in self.H.shape)


def _rng(seed, k=0):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed).spawn(k + 1)[k]))


def gaussian_psf(q, sigma):
    """Gaussian sampled on the integer grid centred at p, truncated to q, sum 1."""
    q = tuple(int(v) for v in q)
    sigma = tuple(float(s) for s in sigma)
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) - (n - 1) / 2 for n in q], indexing="ij")
    e = np.zeros(q, dtype=np.float64)
    for g, s in zip(grids, sigma):
        e += g * g / (2.0 * s * s)
    h = np.exp(-e)
    return (h / h.sum()).astype(np.float32)


def gaussian_factors(q, sigma):
    """Per-axis factors of gaussian_psf(q, sigma): 1-D Gaussians, each sum 1 (their outer product is the template)."""
    out = []
    for n, s in zip(q, sigma):
        g = np.arange(int(n), dtype=np.float64) - (int(n) - 1) / 2
        h = np.exp(-g * g / (2.0 * float(s) * float(s)))
        out.append((h / h.sum()).astype(np.float32))
    return out


def ring_psf(q=(31, 31, 21), sigma=(2.0, 2.0, 4.0), ring_r=10.0, ring_w=1.5, ring_amp=0.2, ring_sz=4.0):
    """Gaussian plus a ring in the (axis1, axis2) plane, Gaussian along axis 3; sum 1."""
    q = tuple(int(v) for v in q)
    g1, g2, g3 = np.meshgrid(*[np.arange(n, dtype=np.float64) - (n - 1) / 2 for n in q], indexing="ij")
    gauss = np.exp(-(g1 ** 2 / (2 * sigma[0] ** 2) + g2 ** 2 / (2 * sigma[1] ** 2) + g3 ** 2 / (2 * sigma[2] ** 2)))
    rho = np.sqrt(g1 ** 2 + g2 ** 2)
    ring = ring_amp * np.exp(-((rho - ring_r) ** 2) / (2 * ring_w ** 2)) * np.exp(-(g3 ** 2) / (2 * ring_sz ** 2))
    h = gauss + ring
    return (h / h.sum()).astype(np.float32)


def blobs(shape, n, rng, sigma=(1.0, 3.0), amp=(0.5, 1.0)):
    """Sum of n isotropic Gaussian blobs with uniform centres on a zero background."""
    shape = tuple(int(s) for s in shape)
    grids = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    X = np.zeros(shape, dtype=np.float64)
    for _ in range(n):
        c = [rng.uniform(0, s - 1) for s in shape]
        s = rng.uniform(*sigma)
        a = rng.uniform(*amp)
        d2 = sum((g - ci) ** 2 for g, ci in zip(grids, c))
        X += a * np.exp(-d2 / (2 * s * s))
    return X.astype(np.float32)


def filaments(shape, n, rng, radius=(1.0, 2.0), intensity=(100.0, 1000.0), background=10.0):
    """n tubular filaments along cubic Bezier curves, plus a constant background.

    Each curve has 4 control points uniform in the volume and is sampled every
    0.25 voxel of control-polygon length; a voxel takes the filament intensity
    if it lies within the filament radius of a sample.  Overlaps take the max.
    """
    shape = tuple(int(s) for s in shape)
    X = np.zeros(int(np.prod(shape)), dtype=np.float32)
    strides = np.array([int(np.prod(shape[i + 1:])) for i in range(3)], dtype=np.int64)
    hi = np.array(shape, dtype=np.float64) - 1
    for _ in range(n):
        P = rng.uniform(0.0, 1.0, size=(4, 3)) * hi
        r = rng.uniform(*radius)
        inten = np.float32(rng.uniform(*intensity))
        plen = np.sum(np.linalg.norm(np.diff(P, axis=0), axis=1))
        ns = max(2, int(math.ceil(plen / 0.25)) + 1)
        t = np.linspace(0.0, 1.0, ns)[:, None]
        pts = ((1 - t) ** 3) * P[0] + 3 * ((1 - t) ** 2) * t * P[1] + 3 * (1 - t) * t * t * P[2] + (t ** 3) * P[3]
        R = int(math.ceil(r))
        o = np.arange(-R, R + 1)
        off = np.stack(np.meshgrid(o, o, o, indexing="ij"), axis=-1).reshape(-1, 3)
        base = np.rint(pts).astype(np.int64)
        vox = (base[:, None, :] + off[None, :, :]).reshape(-1, 3)
        dif = vox - np.repeat(pts, off.shape[0], axis=0)
        ok = (np.einsum("ij,ij->i", dif, dif) <= r * r)
        ok &= np.all((vox >= 0) & (vox <= hi.astype(np.int64)), axis=1)
        flat = np.unique(vox[ok] @ strides)
        X[flat] = np.maximum(X[flat], inten)
    X += np.float32(background)
    return X.reshape(shape)


def observe(X, H, rng, noise="poisson", sigma=0.0):
    """Y = X (*) H + N (Eq. 3): full-size blur by library FFT convolution, then noise."""
    from scipy.signal import fftconvolve
    B = fftconvolve(X.astype(np.float64), H.astype(np.float64), mode="full")
    B = np.maximum(B, 0.0)
    if noise == "poisson":
        Y = rng.poisson(B).astype(np.float32)
    elif noise == "gauss":
        Y = (B + rng.normal(0.0, sigma, size=B.shape)).astype(np.float32)
    elif noise == "none":
        Y = B.astype(np.float32)
    else:
        raise ValueError(noise)
    return Y


def blobs2d(seed=0):
    r = _rng(seed, 0)
    X = blobs((64, 64), 20, r)
    H = gaussian_psf((7, 7), (1.5, 1.5))
    Y = observe(X, H, r, noise="gauss", sigma=0.01)
    return Problem("blobs2d", X, H, Y, 50, {"noise": "gauss 0.01"})


def fil3d(seed=0, shape=(256, 256, 64), q=(15, 15, 11), sigma=(1.5, 1.5, 3.0), n=40, K=100):
    r = _rng(seed, 1)
    X = filaments(shape, n, r)
    H = gaussian_psf(q, sigma)
    Y = observe(X, H, r, noise="poisson")
    return Problem("fil3d", X, H, Y, K, {"noise": "poisson", "filaments": n})


def scaled_fil3d(shape, q, seed=0, K=20):
    """Filament volume of any size with the fil3d density (40 per 256x256x64)."""
    n = max(1, int(round(40 * np.prod(shape) / (256 * 256 * 64))))
    r = _rng(seed, 7)
    X = filaments(shape, n, r)
    H = gaussian_psf(q, tuple(max(0.8, (v - 1) / 5.0) for v in q))
    Y = observe(X, H, r, noise="poisson")
    return Problem("fil3d_%s" % "x".join(map(str, shape)), X, H, Y, K, {"noise": "poisson", "filaments": n})


def grad3d(seed=0, B=4, shape=(128, 128, 64), q=(11, 11, 9), sigma=(1.5, 1.5, 3.0)):
    r = _rng(seed, 2)
    Xs = np.stack([filaments(shape, 10, r) for _ in range(B)])
    H = gaussian_psf(q, sigma)
    return Xs, H, sigma


def ring3d(seed=0, K=100):
    r = _rng(seed, 3)
    X = filaments((512, 512, 128), 320, r)
    H = ring_psf()
    Y = observe(X, H, r, noise="poisson")
    return Problem("ring3d", X, H, Y, K, {"noise": "poisson", "filaments": 320})


def scaled_ring3d(shape, seed=0, K=100):
    """Filament volume of any size at the ring3d density (320 per 512x512x128) with the full
    31x31x21 Gaussian-plus-ring template and Poisson noise."""
    n = max(1, int(round(320 * np.prod(shape) / (512 * 512 * 128))))
    r = _rng(seed, 9)
    X = filaments(shape, n, r)
    H = ring_psf()
    Y = observe(X, H, r, noise="poisson")
    return Problem("ring3d_%s" % "x".join(map(str, shape)), X, H, Y, K, {"noise": "poisson", "filaments": n})


def batch64_shapes(seed=0, count=64):
    """Per-volume (m, q, sigma) of the uneven batch."""
    r = _rng(seed, 4)
    out = []
    for _ in range(count):
        m = (int(r.integers(32, 257)), int(r.integers(32, 257)), int(r.integers(16, 129)))
        q = tuple(int(2 * r.integers(2, 11) + 1) for _ in range(3))   # odd in [5, 21]
        s = tuple(float(r.uniform(0.8, 4.0)) for _ in range(3))
        out.append((m, q, s))
    return out


def batch64(seed=0, count=64, K=200):
    shapes = batch64_shapes(seed, count)
    r = _rng(seed, 5)
    probs = []
    for i, (m, q, s) in enumerate(shapes):
        n = max(1, int(round(40 * np.prod(m) / 4194304)))
        X = filaments(m, n, r)
        H = gaussian_psf(q, s)
        Y = observe(X, H, r, noise="poisson")
        probs.append(Problem("batch64_%d" % i, X, H, Y, K, {"noise": "poisson", "filaments": n}))
    return probs


def integer_case(m, q, seed=0, lo=-3, hi=3):
    """Small integer-valued X and H: every sum is exact in FP64 (and FP32 while < 2^24)."""
    r = _rng(seed, 6)
    X = r.integers(lo, hi + 1, size=tuple(m)).astype(np.float32)
    H = r.integers(-2, 3, size=tuple(q)).astype(np.float32)
    return X, H


def random_case(m, q, seed=0, positive=False):
    """Uniform random X (m) and H (q) and R (m + q - 1), float32."""
    r = _rng(seed, 8)
    lo = 0.0 if positive else -1.0
    X = r.uniform(lo, 1.0, size=tuple(m)).astype(np.float32)
    H = r.uniform(lo, 1.0, size=tuple(q)).astype(np.float32)
    R = r.uniform(-1.0, 1.0, size=tuple(a + b - 1 for a, b in zip(m, q))).astype(np.float32)
    return X, H, R


WORKLOADS = {
    "blobs2d": blobs2d,
    "fil3d": fil3d,
    "ring3d": ring3d,
}

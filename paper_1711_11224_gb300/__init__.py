"""cdv: direct-convolution deconvolution on GB300 (sm_103a).

The hot path of "Properties on n-dimensional convolution for image
deconvolution": the full n-D convolution (Property 1), its adjoint as a
cropped convolution with the flipped template (Property 2), and the
projected-gradient NNLS iteration built from the two (Steps 1-3, Eq. 6).
All arithmetic runs in libcdv.so (hand-written CUDA, C ABI in include/cdv.h);
this package marshals torch tensors into it.
"""
from ._binding import CdvError, load  # noqa: F401
from .plan import BatchPlan, Plan  # noqa: F401

__all__ = ["Plan", "BatchPlan", "CdvError", "load", "conv", "ConvFn"]


def __getattr__(name):
    if name in ("conv", "ConvFn"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)

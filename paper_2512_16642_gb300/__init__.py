"""GB300 data-space Hessian library: Green functions by finite differences with an on-the-fly
transform, per-frequency Gram Hessians, resident Cholesky factors and multi-source deblurring,
all in CUDA kernels behind the C ABI of include/egh.h.  `egh` is the ctypes binding."""
from . import egh  # noqa: F401
from .egh import Context, EghError  # noqa: F401

__all__ = ["egh", "Context", "EghError"]

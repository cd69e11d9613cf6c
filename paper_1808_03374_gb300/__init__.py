"""GB300 library for the top-k principal components of 2-bit-packed genotype
matrices by thick-restarted Golub-Kahan-Lanczos bidiagonalisation
(Chen, Noack, Edelman, arXiv:1808.03374, section 3).

The compute path is libgkl.so (CUDA, sm_103a) behind the C ABI of
include/gkl.h; ``gkl`` is its ctypes binding.
"""
from .build import build  # noqa: F401

__all__ = ["build"]

"""GB300-native ringing-free FFT homogenisation solver (arXiv 2207.10657).

The compute path is librve.so (CUDA, sm_103a) behind the C ABI declared in
include/rve.h; ``binding`` mirrors that ABI with ctypes and ``solver`` wraps
it for torch tensors.  Build with ``paper_2207_10657_gb300.build.build()``.
"""
from . import binding  # noqa: F401
from .driver import LoadPathDriver  # noqa: F401
from .solver import Phase, RVEBatch, RVESolver, make_opts  # noqa: F401

__all__ = ["binding", "LoadPathDriver", "Phase", "RVEBatch", "RVESolver", "make_opts"]

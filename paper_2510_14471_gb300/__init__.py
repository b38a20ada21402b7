"""GB300 (sm_103a) GLS estimation of SUR models by PCG-Aug.

The compute path is the CUDA library ``libglmsur.so`` (C ABI in
include/glm_sur.h); this package is its thin Python binding.  There is no CPU
fallback: calls fail when the library is missing.
"""
from . import _lib
from ._lib import GlmSurError, GlmSurOpts, lib, STATUS_NAMES

__all__ = ["GlmSur", "SolveResult", "GlmSurError", "GlmSurOpts", "lib", "STATUS_NAMES", "_lib"]


def __getattr__(name):
    if name in ("GlmSur", "SolveResult"):
        from . import sur
        return getattr(sur, name)
    raise AttributeError(name)

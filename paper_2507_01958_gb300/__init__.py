"""GB300 (sm_103a) solver for time-dependent variational mean field games with
the parallel-in-time preconditioner of arXiv 2507.01958.

The compute path is the C-ABI library libmfg_gb300.so (include/mfg.h); this
package holds its build script and a thin ctypes binding.  Importing the
binding without the built library raises: there is no CPU fallback.
"""
from .build import build  # noqa: F401


def lib():
    """The ctypes binding (loads libmfg_gb300.so; raises if it is missing)."""
    from . import _lib
    return _lib

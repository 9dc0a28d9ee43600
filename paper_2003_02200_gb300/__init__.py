"""GB300 (sm_103a) total viewshed by the sDEM method (arXiv 2003.02200).

The computation runs in ``libtvs.so`` (hand-written CUDA kernels behind the C
ABI of ``include/tvs.h``); this package is its ctypes binding.  Importing the
package does not load the library: the first call that needs it does, and
raises if the library cannot be built or loaded.  There is no CPU fallback.
"""
from ._binding import (Context, TvsError, count_evals, declared_functions, direction, lib_path,  # noqa: F401
                       load)
from ._build import build  # noqa: F401

__all__ = ["Context", "TvsError", "build", "count_evals", "declared_functions", "direction", "lib_path",
           "load"]

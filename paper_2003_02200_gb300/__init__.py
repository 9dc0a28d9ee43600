"""GB300 (sm_103a) total viewshed by the sDEM method (arXiv 2003.02200).

The computation runs in ``libtvs.so`` (hand-written CUDA kernels behind the C
ABI of ``include/tvs.h``); this package is its ctypes binding.  Importing the
package does not load the library: the first call that needs it does, and
raises if the library cannot be built or loaded.  There is no CPU fallback.
"""
from ._binding import (Batch, Context, Server, TvsError, count_evals, count_point_evals,  # noqa: F401
                       declared_functions, direction, lib_path, load, sweep_check, sweep_stats,
                       total_viewshed_device_noalloc)
from ._build import build  # noqa: F401

__all__ = ["Batch", "Context", "Server", "TvsError", "build", "count_evals", "count_point_evals", "declared_functions",
           "direction", "lib_path", "load", "sweep_check", "sweep_stats",
           "total_viewshed_device_noalloc"]

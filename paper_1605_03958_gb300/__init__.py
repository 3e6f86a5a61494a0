"""GB300 (sm_103a) split-step Crank-Nicolson solver of the 3D Gross-Pitaevskii equation.

The compute path is the CUDA library libgp_sscn.so behind the C ABI in
include/gp.h; this package is its ctypes binding (``gp``).  Importing the package
loads the library and fails loudly when it has not been built: there is no CPU
fallback.
"""
from . import gp
from .gp import (GPError, Pool, Solver, gp_create, gp_create_on, gp_density1d, gp_density2d,
                 gp_destroy, gp_get_g, gp_get_info, gp_get_psi, gp_get_timing, gp_init_gaussian,
                 gp_last_error, gp_observables, gp_set_g, gp_set_psi, gp_set_timing,
                 gp_step_imag, gp_step_real, gp_strerror, gp_sync, gp_workspace_bytes,
                 make_params)

gp.load_library()

__all__ = ["gp", "GPError", "Pool", "Solver", "make_params", "gp_create", "gp_create_on", "gp_destroy",
           "gp_workspace_bytes", "gp_init_gaussian", "gp_set_psi", "gp_get_psi", "gp_step_imag",
           "gp_step_real", "gp_set_g", "gp_get_g", "gp_observables", "gp_density1d",
           "gp_density2d", "gp_sync", "gp_set_timing", "gp_get_timing", "gp_get_info",
           "gp_last_error", "gp_strerror"]

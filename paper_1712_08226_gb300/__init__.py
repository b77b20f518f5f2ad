"""GB300 (sm_103a) generalized-Hopf primal-dual solver.

The compute path is the CUDA library ``libhopf_gb300.so`` (C ABI declared in
include/hopf.h); this package only marshals arguments into it.  Importing the
package does not load the library; the first call does, and fails loudly if
the library has not been built (``python -m paper_1712_08226_gb300.build``).
"""
from .api import (BALL, BOX, FP32, FP64, LEFT_RIEMANN, TRAPEZOID, SIMPSON, LEFT_FIXED, STATUS, VARS_INITIAL,  # noqa: F401
                  VARS_TERMINAL, HopfError,
                  Options, System, last_profile, node_table, time_to_reach, trajectory, value, value_stacked)

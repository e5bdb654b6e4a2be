"""GB300 (sm_103a) multilevel primal-dual Wasserstein-1 solver.

The computation lives in libw1.so (CUDA C++, C ABI in include/w1.h); this
package is its thin Python binding.  See w1.Plan for the solve entry point.
"""
from .w1 import (NORM_L1, NORM_L2, NORM_LINF, Mixed, Options, Plan, Server, Stats, W1Error,  # noqa: F401
                 autotune_level, cp_steps, cp_steps3d, default_options, lib, prolong, prolong3d, restrict,
                 restrict3d, solve3d, state_stats, status_string)

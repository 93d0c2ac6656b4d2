"""B300-native (sm_103a) Lindblad steady-state and low-spectrum library.

The compute lives in liblindblad.so (CUDA kernels + C ABI, include/lindblad.h); this
package is its thin binding.  Importing does not load the library; the first call does,
and raises if it has not been built (python -m paper_2608_30860_b300.build).
"""
from .lindblad import (LB_APPLY_FORM_M, LB_APPLY_HERMITIAN, LB_APPLY_SCHUR, LB_PREC_FP64, LB_PREC_MIXED, LB_ROUTE_AUTO,
                       LB_ROUTE_EIG, LB_ROUTE_SCHUR, Handle, LbInfo, LbOpts, LindbladError, default_opts,
                       implicit_euler, jump_apply, lb_kernel_stats, lb_launch_count, lb_set_profiling,
                       lb_test_bounded_wait, batched_tune, LB_TILE_BUCKETS, LB_TILE_SHAPES, TILE_NAMES,
                       lindblad_batched_workspace_bytes, lindblad_destroy, lindblad_setup,
                       lindblad_workspace_bytes, lindbladian_apply, lindbladian_apply_noalloc, load_library,
                       low_spectrum, pack_batch, phi_apply, resolvent_apply, resolvent_solve, steady_state,
                       steady_state_adjoint, steady_state_batched, steady_state_gmres, unpack_batch)

__all__ = ["LB_APPLY_FORM_M", "LB_APPLY_HERMITIAN", "LB_APPLY_SCHUR", "LB_PREC_FP64", "LB_PREC_MIXED", "LB_ROUTE_AUTO",
           "LB_ROUTE_EIG", "LB_ROUTE_SCHUR", "Handle", "LbInfo", "LbOpts", "LindbladError", "default_opts",
           "implicit_euler", "jump_apply", "lb_kernel_stats", "lb_launch_count", "lb_set_profiling",
           "lb_test_bounded_wait", "batched_tune", "LB_TILE_BUCKETS", "LB_TILE_SHAPES", "TILE_NAMES",
           "lindblad_batched_workspace_bytes", "lindblad_destroy", "lindblad_setup", "lindblad_workspace_bytes",
           "lindbladian_apply", "lindbladian_apply_noalloc", "load_library", "low_spectrum", "pack_batch",
           "phi_apply", "resolvent_apply", "resolvent_solve", "steady_state", "steady_state_adjoint",
           "steady_state_batched", "steady_state_gmres", "unpack_batch"]

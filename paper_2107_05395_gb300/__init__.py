"""paper_2107_05395_gb300 -- shared-LHS batched tridiagonal / pentadiagonal solves
for GB300 (sm_103a).

Many systems A x_m = b_m share one banded matrix A (the setting of "A Batched GPU
Methodology for Numerical Solutions of Partial Differential Equations", sections
2-4).  A is factorised once in FP64 on the host; one device copy of its factors
is staged per CTA and broadcast; every right-hand side, stored interleaved
(element (i, m) at i*ld + m, Fig. 2), is swept forward and back by hand-written
CUDA kernels behind the C ABI in ``include/sbsolve.h``.

This package is the Python side of that ABI: ctypes marshalling only.  Build the
library with ``python -m paper_2107_05395_gb300.build``.
"""
from .autograd import SharedLHSRollout  # noqa: F401,E402
from ._lib import (  # noqa: F401
    SB_ERR_ALLOC, SB_ERR_CUDA, SB_ERR_INVALID_ARG, SB_ERR_SINGULAR, SB_ERR_UNSUPPORTED,
    SB_F32, SB_F64, SB_OK, SIGNATURES, MATRIX_KINDS, Factor, SbError, lib, sb_build_matrix,
    sb_factor_info,
    sb_factor_shared_penta, sb_factor_shared_tri, sb_factor_shared_tri_periodic, sb_factor_shared_penta_periodic, sb_last_error, sb_solve_batched,
    sb_solve_batched_adjoint, sb_solve_batched_ex, sb_version, SB_ARITH_NATIVE, SB_ARITH_DF32,
    Shape, SB_ALGO_SEQUENTIAL, SB_ALGO_PARTITIONED, SB_ALGO_STAGED, SB_ALGO_TWO_ENDED, sb_autotune, sb_shape_get, sb_shape_set, Stepper, sb_stepper_create, sb_stepper_run, sb_stepper_run_coarsening, sb_stepper_set_forcing, sb_stepper_run_forced, sb_stepper_refined_workspace_bytes, sb_stepper_run_refined,
    sb_refine_workspace_bytes, sb_solve_batched_refined, sb_solve_batched_groups,
    sb_solve_batched_refined_noalloc, sb_rollout_workspace_bytes, sb_rollout_forward,
    sb_rollout_backward, sb_host_workspace_bytes, sb_solve_batched_host, sb_device_timeouts, sb_measure_rates,
)

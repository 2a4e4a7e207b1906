"""Polynomial-preconditioned FISTA for multi-coil SENSE on GB300 (sm_103a).

The compute path is libpp.so (CUDA C++ behind the C ABI in include/pp.h);
this package holds its build script and a ctypes binding with the same
function names.  PyTorch supplies device memory and streams only.
"""
from .binding import (  # noqa: F401
    PP_CARTESIAN, PP_NONCARTESIAN, PP_NONCARTESIAN_TOEPLITZ, PPError, Plan, lib, pp_adjoint_apply, pp_adjoint_apply_static, pp_fista_solve, pp_fista_solve_prox,
    pp_forward_apply, pp_last_error, pp_normal_apply, pp_plan_create, pp_plan_destroy,
    pp_plan_scale, pp_plan_set_scale, pp_plan_mu, pp_plan_sizes, pp_plan_tuning, pp_plan_set_tuning, pp_poly_apply, pp_poly_coeffs_l2, pp_poly_coeffs_cheb, pp_poly_coeffs_wl2, pp_poly_max_zp,
    pp_prox_l1_haar, pp_prox_l1_db4, pp_prox_llr, pp_profile_normal, pp_selftest_wait, SolveResult,
    Batch, pp_batch_create, pp_batch_destroy, pp_batch_offsets, pp_batch_scales, pp_batch_set_scales,
    pp_batch_tile, pp_batch_set_tile, pp_batch_forward_apply, pp_batch_adjoint_apply, pp_batch_normal_apply,
    pp_batch_fista_solve, pp_batch_unrolled_forward, pp_batch_unrolled_backward,
)
from .autograd import UnrolledPFISTA, unrolled_pfista  # noqa: F401
from .admm import coil_group_prox, consensus_admm, groups_of_rank  # noqa: F401

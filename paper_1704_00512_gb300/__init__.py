"""GB300-native sparse Chebyshev matrix functions (the CheSS method, arXiv:1704.00512).

The computation lives in libcheb.so (CUDA, sm_103a) behind the C ABI of
include/cheb.h.  This package is its thin Python binding (``_lib``, same names as
the C entry points) plus the solve sequences (``solve``) that chain those calls.
"""
from ._lib import (  # noqa: F401
    BF16, ERFC, F32, F64, F64X, FERMI, INTERVAL, PENALTY, POWER, BatchedPlan, Bsr, ChebError, Plan, bounds, coeffs,
    block_diag, decode_mu_batch, decode_mu_result, expand, expand_batched, newton_schulz_isqrt, expand_workspace_size, plan_resident_info, plan_col_info, plan_col_lists, plan_lists, set_plan_builder, ssf_export, ssf_import, penalty_check, series_value, mu_nodes, lagrange_weights, bounds_spd, bounds_warm, launch_count, load, masked_product, mu_search, mu_search_noalloc, newton_schulz,
    pattern_build, penalty_trace, restrict, scale, tile_shapes, trace, transpose, lincomb, mlp_param_count,
    mlp_init, mlp_forward, mlp_loss, mlp_backward, mlp_adam, mlp_features,
)

"""Nested-dissection selected inversion of contour-integrated density matrices on GB300.

The compute path lives in libndsi.so (C ABI, include/ndsi.h); this package holds its build script
(`build`) and the ctypes binding (`ndsi`).
"""
from .ndsi import (  # noqa: F401
    NdsiError, load, ndsi_default_options, ndsi_poles, ndsi_analyze, ndsi_plan_info,
    ndsi_plan_export, ndsi_factor_poles, ndsi_selinv, ndsi_density, analyze_system,
    NDSI_PREC_FP64, NDSI_PREC_SPLIT, EXPORTED_SYMBOLS, ndsi_profile_enable, ndsi_profile_read,
    ndsi_residue_sum_static, ndsi_find_mu, ndsi_mu_features, ndsi_mlp_init, ndsi_mlp_forward,
    ndsi_mlp_grad, ndsi_mlp_train, NDSI_MLP_PARAMS, analyze_batched, ndsi_density_batched,
    ndsi_graph_enable, ndsi_graph_info, ndsi_autotune, ndsi_density_energy, ndsi_dos, ndsi_factors_solve, ndsi_eigenstates, ndsi_mu_search, ndsi_mu_search_batched, ndsi_find_mu_batched, ndsi_plan_check, ndsi_density_poles, ndsi_pole_shard, ndsi_fp64_peak,
    ndsi_density_batched_poles,
)

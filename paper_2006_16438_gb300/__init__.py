"""GB300 (sm_103a) implementation of the CP-ARLS-LEV sampled least-squares step
(Larsen & Kolda, "Practical Leverage-Based Sampling for Low-Rank Tensor
Decomposition").

The computation lives in the CUDA library ``libcpa.so`` behind the C ABI of
``include/cpa.h``; :mod:`.binding` is its argument-marshalling Python layer.
Importing this package does not load the library; the first call does (and builds it
with nvcc if needed).
"""
from .binding import (  # noqa: F401
    Index, Result, CpaError, load, library_path, default_options,
    cpa_index_build, cpa_index_export, cp_arls_lev, cp_arls_lev_coo, cpa_mode_update, cp_als, Batch,
    cpa_philox4x64, cpa_leverage, cpa_leverage_noalloc, cpa_cdf, cpa_skrp_lev, cpa_sampled_mttkrp, cpa_solve, cpa_fit,
    cpa_fit_terms,
    cpa_fit_sample, cpa_fit_estimate, FitSample, cpa_rrf_init,
    EXPORTED,
)

"""GB300 library for the conditional draw of beta in the CG-accelerated Gibbs
sampler of Nishimura & Suchard (prior-preconditioned conjugate gradient).

The compute runs in the CUDA library ``_pcg_beta.so`` (C ABI in
``include/pcg_beta.h``); this package is its thin Python binding plus the
seeded input generator (``inputs``) and the autograd wrapper (``autograd``).
"""
from ._native import (  # noqa: F401
    ADJ, PCG_BADARG, PCG_BREAKDOWN, PCG_CUDA, PCG_MAXITER, PCG_NONFINITE, PCG_OK, PCG_TIMEOUT,
    PREC, PRECOND, STATUS_NAMES, STOP, Context, DeviceDesign, DrawResult, PcgError, exported_symbols,
    load_library, pcg_adjoint, pcg_build_rhs, pcg_check_design, pcg_ctx_create, pcg_ctx_destroy,
    pcg_draw_beta, pcg_draw_beta_batched, pcg_draw_beta_uneven, pcg_last_error, pcg_phi_mul,
    pcg_last_kernel_launches, pcg_profile_count, pcg_profile_entry, pcg_profile_reset,
    pcg_solve, profile_table, pcg_phi_mul_noalloc, NOALLOC_MAX_N, pcg_set_unshrunk,
    pcg_tiled_plan_applies, pcg_draw_beta_lsqr, pcg_gibbs_step, GibbsState)

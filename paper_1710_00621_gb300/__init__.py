"""GB300 (sm_103a) Wiener-filter / constrained-realization solver for multi-resolution
CMB component separation with the pseudo-inverse preconditioner of Seljebotn et al.
(arXiv:1710.00621).

The compute path is the C-ABI library ``libcmbws.so`` (hand-written CUDA kernels); this
package is a thin ctypes binding with the same call names (``cmbws_plan_grid``,
``cmbws_sht_synth``, ``cmbws_sht_analysis``, ``cmbws_model_create``, ``cmbws_apply_A``,
``cmbws_apply_precond``, ``cmbws_rhs``, ``cmbws_cg_solve``, ``cmbws_cr_sample``, ``cmbws_grad_terms``; the
autograd wrapper is in ``autodiff``).  PyTorch only supplies
device memory and streams.  There is no CPU fallback: loading fails loudly when the
library has not been built.
"""
from .binding import (  # noqa: F401
    CMBWS_3XTF32,
    CMBWS_DRAW_NORMAL,
    CMBWS_DRAW_UNIFORM,
    CMBWS_FP32,
    CMBWS_FP32X2,
    CMBWS_FP64,
    CMBWS_GRID_GL,
    CMBWS_GRID_HEALPIX,
    CMBWS_TF32,
    CMBWS_VCYCLE_BASIC,
    CMBWS_VCYCLE_OPTIMIZED,
    CmbwsError,
    CgOpts,
    CgReport,
    Grid,
    Model,
    cmbws_apply_A,
    cmbws_apply_M_add,
    cmbws_apply_M_diag,
    cmbws_apply_precond,
    cmbws_cg_solve,
    cmbws_cg_solve_batched,
    cmbws_cr_rhs,
    cmbws_cr_sample,
    cmbws_draw,
    cmbws_grad_terms,
    cmbws_grid_destroy,
    cmbws_grid_info,
    cmbws_grid_rings,
    cmbws_model_add_mask_precond,
    cmbws_model_create,
    cmbws_model_destroy,
    cmbws_model_info,
    cmbws_model_merge_precond,
    cmbws_model_set_graphs,
    cmbws_model_set_vcycle,
    cmbws_plan_grid,
    cmbws_powerlaw_mixing,
    cmbws_profile_enable,
    cmbws_profile_read,
    cmbws_project,
    cmbws_rhs,
    cmbws_sht_analysis,
    cmbws_sht_analysis_noalloc,
    cmbws_sht_synth,
    exported_symbols,
    library_path,
    load_library,
)

"""GB300 (sm_103a) Cholesky factorization, solution and inversion in
Rectangular Full Packed Format.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/rfp.h``); this package only marshals arguments to it.  There is no
CPU fallback: calling any entry point without the built library raises.
"""
from .binding import (  # noqa: F401
    DEFAULT_LIB,
    Library,
    RfpError,
    library,
    rfp_dpack,
    rfp_dpftrf,
    rfp_dpftri,
    rfp_dpftrs,
    rfp_dunpack,
    rfp_kernel_launches,
    rfp_layout,
    rfp_spack,
    rfp_spftrf,
    rfp_spftri,
    rfp_spftrs,
    rfp_stage_timing,
    rfp_stage_times,
    rfp_sunpack,
    rfp_ssyrk_tc,
    RFP_PREC_BF16,
    RFP_PREC_TF32,
    RFP_PREC_FP32,
    RFP_PREC_TF32X3,
    RFP_PREC_BF16X6,
    rfp_dpfsv_mixed,
    rfp_dpfsv_mixed_workspace,
    mixed_status,
)
from .flops import pftrf_flops, pftri_flops, pftrs_flops, pack_bytes  # noqa: F401

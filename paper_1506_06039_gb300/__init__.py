"""moco on GB300: the translation search of "moco: Fast Motion Correction for
Calcium Imaging" (arXiv 1506.06039, Section 2) as hand-written sm_103a CUDA
behind a C ABI (include/moco.h), with a thin ctypes binding.

Importing the package loads nothing; the CUDA library is loaded on the
first call into the binding and must have been built first
(paper_1506_06039_gb300.build.build()).
"""
from .binding import (  # noqa: F401
    EXPORTS, PEAK_DP2A, PEAK_FP32_FMA, FrameStream, MocoError, Plan, TEMPLATE_F32, TEMPLATE_U16, XCORR_AUTO,
    XCORR_DIRECT_BF16X3, XCORR_FFT_FP32, moco_alu_peak, moco_jitter_noalloc, moco_align_host, moco_align_stack, moco_apply_shifts, moco_cost_backward, moco_cost_surface,
    moco_plan, moco_plan_destroy, moco_plan_query, moco_plan_status, moco_profile_enable, moco_profile_read,
    moco_selftest_wait, moco_set_template, moco_softmin, moco_softmin_grad, moco_status_string,
)

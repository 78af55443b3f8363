"""B300-native direct solver for the 2D type-II inverse NUDFT (HSS face-splitting + URV).

Public API: NudftHSS (build / factor / solve / apply / grad / plsqr / checkpoint / save / load /
info / kstats; fadi=True builds the 1D factors by fADI + interpolative decomposition), lstsq
(differentiable solve), run_batched and build_batched / solve_batched (many uneven problems),
exact_apply, psi_eval, fadi_plan (the host-side shift plan), the dense building blocks la_gemm /
la_qr / la_qr_apply / la_tsvd, peak_fma, and the operator constants of include/nudft2_hss.h.  All
arithmetic runs in the CUDA library libnudft2_hss.so.
"""
from .binding import (  # noqa: F401
    EXACT_ADJ, EXACT_FWD, FAST_ADJ, FAST_FWD, FP64, MIXED, PINV, PINV_ADJ, LIB_PATH, NudftError, NudftHSS, lib,
    build_batched, exact_apply, fadi_plan, la_gemm, la_qr, la_qr_apply, la_tsvd, lstsq, peak_fma, psi_eval, run_batched, solve_batched,
)

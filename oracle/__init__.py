"""CPU FP64 oracle for the 2D type-II inverse NUDFT least-squares solve.

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the library.  Every function is pinned by the
non-GPU tests in tests/test_oracle_pins.py (and tests/test_oracle_fadi.py for the fADI + ID
construction of the 1D HSS in ``oracle.fadi_oracle``).  Shares no code with the CUDA path.
"""
from .nudft_oracle import (  # noqa: F401
    normal_cg, lstsq_grad_rows, nudft_1d, nudft_matrix, forward, adjoint, householder_qr, apply_qh, apply_q, back_substitute,
    lstsq, cgls, dft_matrix, tilde_1d, tilde_2d, idft2, relres, relerr, forward_substitute_h, pinv_adjoint,
    lstsq_grad,
)

"""GB300 (sm_103a) variable-block CSR operator library.

Hot path: Y = alpha H X + beta Y on a variable-block sparse operator whose
(i, j) block is a dense b_i x b_j matrix, its adjoint (Eq. 1 of the paper),
the pattern-sampled gradient product, mixed-precision block products and the
Chebyshev recurrence of the kernel polynomial method. All arithmetic runs in
hand-written CUDA kernels behind the C ABI in include/vbcsr.h.
"""
from ._lib import VBCSRError, lib  # noqa: F401
from .matrix import VBCSR, kpm_dos, kpm_gap  # noqa: F401

__all__ = ["VBCSR", "VBCSRError", "lib"]
from .autograd import VBCSRMatmul, chebyshev_moments, vbcsr_matmul  # noqa: F401,E402

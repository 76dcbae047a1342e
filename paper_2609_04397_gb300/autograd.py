"""Differentiable products on a VBCSR operator (torch.autograd.Function).

* ``vbcsr_matmul(H, values, X)``  Y = H(values) X;  dX = H^T dY (adjoint
  kernel, Eq. 1), dvalues = pattern-sampled dY X^T (block-SDDMM kernel).
* ``chebyshev_moments(H, values, R, n_moments, ckpt_every, c=, d=)``  the
  moments mu_n = <R, T_n(H~) R> / (N k) of the kernel polynomial method
  (Sec. V) for H~ = (H - c I) / d, H holding ``values``; the shift and scale
  run in the library (vbcsr_shift_scale), and the backward pass runs the
  adjoint recurrence in the library, recomputing the Chebyshev vectors from
  checkpoint pairs (t_m, t_m+1) stored every ``ckpt_every`` steps, and divides
  by d there.

The gradient flows to every stored value independently (a mirrored block of
a symmetric operator is a separate parameter).
"""
import ctypes

import numpy as np
import torch

from ._lib import check, lib
from .matrix import VBCSR, _prec, _stream


class _Matmul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, X, H: VBCSR, precision):
        H.set_values(values.detach())
        Y = H.spmm(X.detach(), precision=precision)
        ctx.save_for_backward(values, X)
        ctx.H, ctx.precision = H, precision
        return Y

    @staticmethod
    def backward(ctx, dY):
        values, X = ctx.saved_tensors
        H = ctx.H
        dY = dY.contiguous()
        H.set_values(values.detach())
        dvalues = dX = None
        if ctx.needs_input_grad[0]:
            dvalues = H.sddmm(dY, X.detach().contiguous())
        if ctx.needs_input_grad[1]:
            dX = H.spmm_adjoint(dY, precision=ctx.precision)
        return dvalues, dX, None, None


# The Function itself: VBCSRMatmul.apply(values, X, H, precision)
VBCSRMatmul = _Matmul


def vbcsr_matmul(H: VBCSR, values: torch.Tensor, X: torch.Tensor, precision="native") -> torch.Tensor:
    """Y = H X with the stored values taken from `values` (packed order)."""
    return _Matmul.apply(values, X, H, precision)


class _Chebyshev(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, R, H: VBCSR, n_moments, ckpt_every, precision, c, d):
        H.set_values(values.detach())
        scaled = (c, d) != (0.0, 1.0)
        if scaled:
            H.shift_scale(c, d)                  # H~ = (H - c I) / d, in the library
        R = R.detach().contiguous()
        mom, ck = H.chebyshev(R, n_moments, ckpt_every=ckpt_every, precision=precision)
        ctx.save_for_backward(values, R, ck if ck is not None else torch.empty(0, device=R.device))
        ctx.H, ctx.M, ctx.E, ctx.precision, ctx.c, ctx.d = H, n_moments, ckpt_every, precision, c, d
        return mom

    @staticmethod
    def backward(ctx, grad_mu):
        values, R, ck = ctx.saved_tensors
        H, M, E = ctx.H, ctx.M, ctx.E
        H.set_values(values.detach())
        if (ctx.c, ctx.d) != (0.0, 1.0):
            H.shift_scale(ctx.c, ctx.d)
        N, k = R.shape
        dv = torch.empty(H.nnz, dtype=torch.float64, device=R.device)
        work = torch.empty((2 + 2 * E) * N * k, dtype=torch.float64, device=R.device)
        g = grad_mu.detach().to(torch.float64).contiguous()
        # dL/dH = dL/dH~ / d: the library divides by d (the shift c drops out)
        check(lib().vbcsr_chebyshev_backward(
            H.handle, k, ctypes.c_void_p(R.data_ptr()), R.stride(0), M, ctypes.c_void_p(g.data_ptr()),
            ctypes.c_void_p(ck.data_ptr() if ck.numel() else None), E, float(ctx.d),
            ctypes.c_void_p(dv.data_ptr()), ctypes.c_void_p(work.data_ptr()), _prec(ctx.precision),
            _stream(H.device)), "vbcsr_chebyshev_backward")
        return dv, None, None, None, None, None, None, None


def chebyshev_moments(H: VBCSR, values: torch.Tensor, R: torch.Tensor, n_moments: int,
                      ckpt_every: int = 10, precision="native", c: float = 0.0, d: float = 1.0) -> torch.Tensor:
    """Differentiable KPM moments mu_n = <R, T_n(H~) R> / (N k) of
    H~ = (H - c I) / d, H holding `values` (packed order). With the default
    c = 0, d = 1 the values are those of H~ itself (spectrum inside [-1, 1]);
    otherwise the library forms H~ from them (vbcsr_shift_scale) and the
    gradient is with respect to the values of H (c and d are constants)."""
    if H.dtype != torch.float64:
        raise TypeError("the Chebyshev recurrence runs on an FP64 operator")
    d = float(d)
    if not (d != 0.0 and np.isfinite(d)):
        raise ValueError(f"d = {d}")
    return _Chebyshev.apply(values, R, H, n_moments, max(1, int(ckpt_every)), precision, float(c), d)

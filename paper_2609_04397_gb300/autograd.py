"""Differentiable products on a VBCSR operator (torch.autograd.Function).

* ``vbcsr_matmul(H, values, X)``  Y = H(values) X;  dX = H^T dY (adjoint
  kernel, Eq. 1), dvalues = pattern-sampled dY X^T (block-SDDMM kernel).
* ``chebyshev_moments(H, values_t, R, n_moments, ckpt_every)``  the moments
  mu_n = <R, T_n(H~) R> / (N k) of the kernel polynomial method (Sec. V) for
  the already shifted and scaled operator H~ = values_t; the backward pass runs
  the adjoint recurrence in the library, recomputing the Chebyshev vectors
  from checkpoint pairs (t_m, t_m+1) stored every ``ckpt_every`` steps.

The gradient flows to every stored value independently (a mirrored block of
a symmetric operator is a separate parameter).
"""
import ctypes

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
    def forward(ctx, values_t, R, H: VBCSR, n_moments, ckpt_every, precision):
        H.set_values(values_t.detach())
        R = R.detach().contiguous()
        mom, ck = H.chebyshev(R, n_moments, ckpt_every=ckpt_every, precision=precision)
        ctx.save_for_backward(values_t, R, ck if ck is not None else torch.empty(0, device=R.device))
        ctx.H, ctx.M, ctx.E, ctx.precision = H, n_moments, ckpt_every, precision
        return mom

    @staticmethod
    def backward(ctx, grad_mu):
        values_t, R, ck = ctx.saved_tensors
        H, M, E = ctx.H, ctx.M, ctx.E
        H.set_values(values_t.detach())
        N, k = R.shape
        dv = torch.empty(H.nnz, dtype=torch.float64, device=R.device)
        work = torch.empty((2 + 2 * E) * N * k, dtype=torch.float64, device=R.device)
        g = grad_mu.detach().to(torch.float64).contiguous()
        check(lib().vbcsr_chebyshev_backward(
            H.handle, k, ctypes.c_void_p(R.data_ptr()), R.stride(0), M, ctypes.c_void_p(g.data_ptr()),
            ctypes.c_void_p(ck.data_ptr() if ck.numel() else None), E, ctypes.c_void_p(dv.data_ptr()),
            ctypes.c_void_p(work.data_ptr()), _prec(ctx.precision), _stream(H.device)),
            "vbcsr_chebyshev_backward")
        return dv, None, None, None, None, None


def chebyshev_moments(H: VBCSR, values_t: torch.Tensor, R: torch.Tensor, n_moments: int,
                      ckpt_every: int = 10, precision="native") -> torch.Tensor:
    """Differentiable KPM moments of H~ (values_t, spectrum inside [-1, 1])."""
    if H.dtype != torch.float64:
        raise TypeError("the Chebyshev recurrence runs on an FP64 operator")
    return _Chebyshev.apply(values_t, R, H, n_moments, max(1, int(ckpt_every)), precision)


def diagonal_mask(H: VBCSR) -> torch.Tensor:
    """1.0 at every stored value on the scalar diagonal (packed order), else 0."""
    import numpy as np
    rb, cb, rp, ci = H.pattern
    r = np.concatenate([[0], np.cumsum(rb.astype(np.int64))])
    c = np.concatenate([[0], np.cumsum(cb.astype(np.int64))])
    rows = np.repeat(np.arange(len(rb)), np.diff(rp))
    off = np.concatenate([[0], np.cumsum(rb[rows].astype(np.int64) * cb[ci])])
    m = np.zeros(int(off[-1]))
    # only blocks whose scalar row and column ranges overlap hold diagonal entries
    hit = np.nonzero((r[rows] < c[ci] + cb[ci]) & (c[ci] < r[rows] + rb[rows]))[0]
    for b in hit:
        i, j = rows[b], ci[b]
        p = np.arange(rb[i])[:, None] + r[i]
        q = np.arange(cb[j])[None, :] + c[j]
        m[off[b]:off[b + 1]] = (p == q).astype(np.float64).ravel()
    return torch.from_numpy(m).to(H.device)


def shift_scale(values: torch.Tensor, diag_mask: torch.Tensor, c: float, d: float) -> torch.Tensor:
    """Packed values of H~ = (H - c I) / d; c and d are constants."""
    return (values - c * diag_mask) / d

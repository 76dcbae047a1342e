"""Comparison helpers for the GPU parity tests.

Tolerances (per result):
* FP64 path: ||Y - Y_ref||_F / ||Y_ref||_F <= 1e-12, and element by element
  |Y - Y_ref| <= 1e-12 * (|H| |X|) + tiny, the scaled forward-error bound of
  a dot product (the products reorder the summation).
* mixed / FP32 paths: the same with 1e-5.
"""
import numpy as np

import oracle

TOL_F64 = 1e-12
TOL_MIXED = 1e-5


def _as_f64(a):
    a = np.asarray(a)
    return a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)


def rel_fro(got, ref):
    d = np.linalg.norm(_as_f64(got) - ref)
    n = np.linalg.norm(ref)
    return d / n if n > 0 else d


def check_elementwise(got, ref, scale, tol):
    got = _as_f64(got)
    bad = np.abs(got - ref) > tol * scale + 1e-300
    assert not bad.any(), (f"{bad.sum()} entries off; worst "
                           f"{np.max(np.abs(got - ref) / np.maximum(scale, 1e-300))}")


def forward_ref(pat, values, X, alpha, beta, Y0):
    ref = oracle.spmm(pat, values, X, alpha, beta, Y0)
    # |alpha| |H| |X| + |beta| |Y0|: the magnitude the rounding errors scale with
    scale = oracle.spmm(pat, np.abs(values), np.abs(X), abs(alpha), 0.0)
    if beta != 0.0 and Y0 is not None:
        scale = scale + abs(beta) * np.abs(Y0)
    return ref, scale


def adjoint_ref(pat, values, X, alpha, beta, Y0):
    ref = oracle.spmm_adjoint(pat, values, X, alpha, beta, Y0)
    scale = oracle.spmm_adjoint(pat, np.abs(values), np.abs(X), abs(alpha), 0.0)
    if beta != 0.0 and Y0 is not None:
        scale = scale + abs(beta) * np.abs(Y0)
    return ref, scale


def sddmm_ref(pat, A, B, alpha, beta, D0):
    ref = oracle.sddmm(pat, A, B, alpha, beta, D0)
    scale = oracle.sddmm(pat, np.abs(A), np.abs(B), abs(alpha), 0.0)
    if beta != 0.0 and D0 is not None:
        scale = scale + abs(beta) * np.abs(D0)
    return ref, scale

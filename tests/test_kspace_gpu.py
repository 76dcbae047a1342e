"""GPU parity of the reciprocal-space sampling of a periodic operator (Eq. 4)
and of the complex block products (the dagger of Eq. 1 a conjugate
transpose) against the oracle, on periodic zinc-blende crystals: one
conventional cell (cutoff beyond half the box: several images per atom
pair) and 2 x 2 x 2 cells (one image per pair)."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as syn
from synthetic.structures import BlockPattern
from _parity import TOL_F64, check_elementwise, rel_fro

pytestmark = pytest.mark.gpu

KPOINTS = ([0.0, 0.0, 0.0], [0.1, 0.2, 0.3], [0.5, 0.5, 0.5], [-0.37, 0.81, 0.05])


def _kspace(w, tau=False):
    from paper_2609_04397_gb300 import VBCSR
    return VBCSR.from_images(w.bsize, w.edge_i, w.edge_j, w.edge_R, w.edge_values,
                             tau=w.tau if tau else None, device="cuda:0")


def _oracle_blocks(w, k, tau=False):
    rb, cb, ptr, cols, vals = oracle.kspace_blocks(w.bsize, w.edge_i, w.edge_j, w.edge_R, w.edge_values, k,
                                                   w.tau if tau else None)
    return BlockPattern(rb, cb, ptr, cols), vals


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", torch.complex128)


@pytest.mark.parametrize("n_cells", [1, 2])
@pytest.mark.parametrize("tau", [False, True])
def test_kpoint_values_match_oracle(n_cells, tau):
    w = syn.zincblende_crystal(n_cells)
    H = _kspace(w, tau)
    assert H.dtype == torch.complex128
    assert not H.get_values().abs().any()           # zero until the first k-point
    vmax = np.abs(w.edge_values).max()
    for k in KPOINTS:
        H.set_kpoint(k)
        pat, ref = _oracle_blocks(w, k, tau)
        assert np.array_equal(H.pattern[2], pat.block_row_ptr)
        assert np.array_equal(H.pattern[3], pat.block_col_idx)
        got = H.get_values().cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-13 * vmax


@pytest.mark.parametrize("schedule", ["persistent", "bucketed"])
@pytest.mark.parametrize("k", [1, 3, 8, 33])
def test_complex_products_match_oracle(k, schedule):
    w = syn.zincblende_crystal(2)
    H = _kspace(w)
    H.set_schedule(schedule)
    kp = [0.13, -0.27, 0.41]
    H.set_kpoint(kp)
    pat, vals = _oracle_blocks(w, kp)
    rng = np.random.default_rng(k)
    X = _crandn(rng, pat.n_cols, k + 1)
    Y0 = _crandn(rng, pat.n_rows, k + 2)
    for alpha, beta in ((1.0, 0.0), (2.0, -0.5), (0.0, 1.5)):
        Yd = _dev(Y0)
        H.spmm(_dev(X)[:, :k], alpha, beta, Yd[:, :k])
        got = Yd.cpu().numpy()
        ref = oracle.spmm_complex(pat, vals, X[:, :k], alpha, beta, Y0[:, :k])
        scale = abs(alpha) * oracle.spmm(pat, np.abs(vals), np.abs(X[:, :k])) + abs(beta) * np.abs(Y0[:, :k])
        assert rel_fro(got[:, :k], ref) <= TOL_F64
        check_elementwise(got[:, :k], ref, scale, TOL_F64)
        assert np.array_equal(got[:, k:], Y0[:, k:])      # columns beyond k untouched
        Yd = _dev(Y0)
        H.spmm_adjoint(_dev(X)[:, :k], alpha, beta, Yd[:, :k])
        ref = oracle.spmm_adjoint_complex(pat, vals, X[:, :k], alpha, beta, Y0[:, :k])
        assert rel_fro(Yd.cpu().numpy()[:, :k], ref) <= TOL_F64
        check_elementwise(Yd.cpu().numpy()[:, :k], ref, scale, TOL_F64)
    H.check()


def test_hermitian_sample_and_adjoint_identity():
    """Symmetric images give a Hermitian O(k): the adjoint product equals the
    forward one to rounding, and <Y, H X> = <H^dagger Y, X> on the GPU."""
    w = syn.zincblende_crystal(1)
    H = _kspace(w)
    H.set_kpoint([0.31, 0.07, -0.44])
    rng = np.random.default_rng(3)
    X = _dev(_crandn(rng, H.shape[1], 4))
    Y = _dev(_crandn(rng, H.shape[0], 4))
    HX, HaX = H.spmm(X), H.spmm_adjoint(X)
    assert torch.allclose(HX, HaX, rtol=0, atol=1e-12 * HX.abs().max().item())
    lhs = torch.vdot(Y.flatten(), HX.flatten())
    rhs = torch.vdot(H.spmm_adjoint(Y).flatten(), X.flatten())
    assert abs(lhs - rhs).item() <= 1e-12 * abs(lhs).item()


def test_complex_epilogue_dot_and_create_from_values():
    """A C128 operator created from packed complex values; the fused epilogue
    Y = alpha H X + beta Y + gamma Z with dot = Re sum(conj(R) .* Y)."""
    from paper_2609_04397_gb300 import VBCSR
    pat = syn.random_pattern(29, 29, (1, 4, 9, 13), 0.2, 5, empty_rows=2, unsorted=True)
    rng = np.random.default_rng(5)
    vals = _crandn(rng, pat.nnz)
    H = VBCSR.from_pattern(pat, vals, torch.complex128, "cuda:0")
    X = _crandn(rng, pat.n_cols, 3)
    Y0, Z, R = (_crandn(rng, pat.n_rows, 3) for _ in range(3))
    Yd = _dev(Y0)
    dot = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    H.spmm_ex(_dev(X), 2.0, -1.0, Yd, gamma=0.5, Z=_dev(Z), R=_dev(R), dot_out=dot)
    ref = oracle.spmm_complex(pat, vals, X, 2.0, -1.0, Y0) + 0.5 * Z
    got = Yd.cpu().numpy()
    assert rel_fro(got, ref) <= TOL_F64
    want = float(np.sum(R.real * got.real + R.imag * got.imag))
    assert abs(dot.item() - want) <= 1e-12 * float(np.sum(np.abs(R) * np.abs(got)))
    assert np.allclose(H.get_values().cpu().numpy(), vals, rtol=0, atol=0)


def test_complex_operator_rejects_what_it_does_not_support():
    from paper_2609_04397_gb300 import VBCSR
    from paper_2609_04397_gb300._lib import VBCSRError
    w = syn.zincblende_crystal(1)
    H = _kspace(w)
    H.set_kpoint([0.1, 0.0, 0.0])
    X = _dev(np.ones((H.shape[1], 2)))
    for prec in ("bf16x2", "df32", "f32"):
        with pytest.raises(VBCSRError, match="UNSUPPORTED"):
            H.spmm(X, precision=prec)
    with pytest.raises(VBCSRError, match="UNSUPPORTED"):
        H.sddmm(X, X)
    real = VBCSR.from_pattern(syn.tiny_multispecies(0).pattern, syn.tiny_multispecies(0).values,
                              torch.float64, "cuda:0")
    with pytest.raises(VBCSRError, match="INVALID_ARG"):
        real.set_kpoint([0.0, 0.0, 0.0])


def test_kpm_moments_of_a_kpoint():
    """The kernel-polynomial pipeline at a reciprocal-space point: Gershgorin
    bounds of the Hermitian O(k), the shift and scale, the Chebyshev moments
    with random-phase vectors and the doubling moments, against the oracle."""
    w = syn.zincblende_crystal(2)
    kp = [0.21, -0.13, 0.34]
    H = _kspace(w)
    H.set_kpoint(kp)
    pat, vals = _oracle_blocks(w, kp)
    lo, hi = oracle.gershgorin_bounds_complex(pat, vals)
    glo, ghi = H.gershgorin()
    assert abs(glo - lo) <= 1e-12 * abs(lo) and abs(ghi - hi) <= 1e-12 * abs(hi)
    c, d = 0.5 * (hi + lo), 1.01 * 0.5 * (hi - lo)
    H.shift_scale(c, d)
    vt = oracle.shift_scale_values_complex(pat, vals, c, d)
    assert np.abs(H.get_values().cpu().numpy() - vt).max() <= 1e-14 * np.abs(vt).max()
    rng = np.random.default_rng(11)
    R = np.exp(2j * np.pi * rng.random((pat.n_rows, 4)))
    ref = oracle.chebyshev_moments_complex(pat, vt, R, 24)
    mom, _ = H.chebyshev(_dev(R), 24)
    assert np.abs(mom.cpu().numpy() - ref).max() <= 1e-12
    mom2 = H.kpm_moments(_dev(R), 24)
    assert np.abs(mom2.cpu().numpy() - ref).max() <= 1e-12

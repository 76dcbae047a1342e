"""Pins for the CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against something the mathematics fixes: a
hand-worked example, dense matrix algebra, SciPy's CSR / BSR products on the
uniform-block special cases (Sec. II.B backend equivalence), symmetry and
adjoint identities, closed forms of the Chebyshev recurrence, and central
finite differences for the gradient.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synthetic as syn
from synthetic.structures import BlockPattern

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hand():
    with open(os.path.join(GOLDEN, "tiny_hand.json")) as f:
        g = json.load(f)
    pat = BlockPattern(np.array(g["row_bsize"]), np.array(g["col_bsize"]),
                       np.array(g["block_row_ptr"]), np.array(g["block_col_idx"]))
    return g, pat, np.array(g["values"], dtype=np.float64)


def test_hand_worked_example():
    g, pat, v = _hand()
    X = np.array(g["X"], dtype=np.float64)
    assert np.array_equal(oracle.to_dense(pat, v), np.array(g["dense_H"], dtype=np.float64))
    assert np.array_equal(oracle.spmm(pat, v, X), np.array(g["HX"], dtype=np.float64))
    Y0 = np.array(g["Y0"], dtype=np.float64)
    assert np.array_equal(oracle.spmm(pat, v, X, 2.0, -1.0, Y0),
                          np.array(g["alpha2_beta_minus1"], dtype=np.float64))
    assert np.array_equal(oracle.spmm_adjoint(pat, v, X), np.array(g["HtX"], dtype=np.float64))
    assert np.array_equal(oracle.sddmm(pat, X, X), np.array(g["sddmm_X_X"], dtype=np.float64))


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_spmm_matches_dense_random_rectangular(seed):
    pat = syn.random_pattern(17, 11, (1, 2, 3, 5, 8), 0.3, seed, empty_rows=3, unsorted=True)
    v = syn.random_values(pat, seed)
    H = oracle.to_dense(pat, v)
    rng = np.random.default_rng(seed)
    for k in (1, 3, 8):
        X = rng.standard_normal((pat.n_cols, k))
        Y0 = rng.standard_normal((pat.n_rows, k))
        for alpha, beta in ((1.0, 0.0), (-0.5, 1.0), (2.0, -1.0), (0.0, 0.7)):
            ref = alpha * (H @ X) + beta * Y0
            got = oracle.spmm(pat, v, X, alpha, beta, Y0)
            assert _rel(got, ref) < 1e-14
            # adjoint against the dense transpose
            Xa = rng.standard_normal((pat.n_rows, k))
            Ya = rng.standard_normal((pat.n_cols, k))
            ref_a = alpha * (H.T @ Xa) + beta * Ya
            assert _rel(oracle.spmm_adjoint(pat, v, Xa, alpha, beta, Ya), ref_a) < 1e-14


def test_beta_zero_does_not_read_y():
    pat = syn.random_pattern(6, 6, (2, 3), 0.5, 3)
    v = syn.random_values(pat, 3)
    X = np.ones((pat.n_cols, 2))
    Y0 = np.full((pat.n_rows, 2), np.nan)
    assert np.isfinite(oracle.spmm(pat, v, X, 1.0, 0.0, Y0)).all()
    assert np.isfinite(oracle.spmm_adjoint(pat, v, np.ones((pat.n_rows, 2)), 1.0, 0.0,
                                           np.full((pat.n_cols, 2), np.nan))).all()


def test_tiny_multispecies_against_dense():
    w = syn.tiny_multispecies(0)
    pat, v = w.pattern, w.values
    X = syn.normal_panel(pat.n_cols, 8, 0)
    H = oracle.to_dense(pat, v)
    assert H.shape == (1300, 1300)
    assert _rel(oracle.spmm(pat, v, X), H @ X) < 1e-14


def _uniform_pattern(n, b, density, seed):
    rng = np.random.default_rng(seed)
    mask = rng.random((n, n)) < density
    np.fill_diagonal(mask, True)
    ptr = np.concatenate([[0], np.cumsum(mask.sum(1))])
    cols = np.concatenate([np.nonzero(mask[i])[0] for i in range(n)])
    return BlockPattern(np.full(n, b), np.full(n, b), ptr, cols)


def test_uniform_b1_is_scipy_csr():
    pat = _uniform_pattern(300, 1, 0.05, 4)
    v = syn.random_values(pat, 4)
    A = sp.csr_matrix((v, pat.block_col_idx, pat.block_row_ptr), shape=(300, 300))
    X = syn.normal_panel(300, 5, 4)
    assert _rel(oracle.spmm(pat, v, X), A @ X) < 1e-14
    assert _rel(oracle.spmm_adjoint(pat, v, X), A.T @ X) < 1e-14


def test_uniform_b8_is_scipy_bsr():
    n, b = 60, 8
    pat = _uniform_pattern(n, b, 0.1, 5)
    v = syn.random_values(pat, 5)
    A = sp.bsr_matrix((v.reshape(-1, b, b), pat.block_col_idx, pat.block_row_ptr),
                      shape=(n * b, n * b))
    X = syn.normal_panel(n * b, 16, 5)
    assert _rel(oracle.spmm(pat, v, X), A @ X) < 1e-14
    assert _rel(oracle.spmm_adjoint(pat, v, X), A.T @ X) < 1e-14
    # the same operator held as b=1 CSR must agree too
    Acsr = A.tocsr()
    assert _rel(oracle.spmm(pat, v, X), Acsr @ X) < 1e-14


def test_symmetric_operator_quadratic_form():
    """X^T H X is symmetric when H = H^T (the generator's H_ji = H_ij^T)."""
    w = syn.tiny_multispecies(0)
    X = syn.normal_panel(w.pattern.n_cols, 8, 0)
    Q = X.T @ oracle.spmm(w.pattern, w.values, X)
    assert np.abs(Q - Q.T).max() < 1e-12 * np.abs(Q).max()
    # and the adjoint equals the forward product for a symmetric H
    assert _rel(oracle.spmm_adjoint(w.pattern, w.values, X), oracle.spmm(w.pattern, w.values, X)) < 1e-14


def test_adjoint_dot_product_identity():
    pat = syn.random_pattern(23, 19, (1, 4, 9, 13), 0.2, 7, empty_rows=2)
    v = syn.random_values(pat, 7)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((pat.n_cols, 4))
    Y = rng.standard_normal((pat.n_rows, 4))
    lhs = np.sum(Y * oracle.spmm(pat, v, X))
    rhs = np.sum(oracle.spmm_adjoint(pat, v, Y) * X)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_sddmm_matches_dense_masked_product():
    pat = syn.random_pattern(13, 9, (1, 4, 9, 13), 0.3, 8, empty_rows=2, unsorted=True)
    rng = np.random.default_rng(8)
    A = rng.standard_normal((pat.n_rows, 7))
    B = rng.standard_normal((pat.n_cols, 7))
    D0 = rng.standard_normal(pat.nnz)
    dense = A @ B.T
    ones = np.ones(pat.nnz)
    mask = oracle.to_dense(pat, ones) > 0
    got = oracle.sddmm(pat, A, B, 0.5, -2.0, D0)
    # scatter the packed result back to dense and compare on the pattern
    G = oracle.to_dense(pat, got)
    G0 = oracle.to_dense(pat, D0)
    assert np.allclose(G[mask], (0.5 * dense - 2.0 * G0)[mask], rtol=0, atol=1e-13)
    # gradient identity: d/dv <Y, H X> = sddmm(Y, X)
    X = rng.standard_normal((pat.n_cols, 3))
    Y = rng.standard_normal((pat.n_rows, 3))
    g = oracle.sddmm(pat, Y, X)
    v = syn.random_values(pat, 8)
    f0 = np.sum(Y * oracle.spmm(pat, v, X))
    e = np.zeros_like(v)
    idx = rng.choice(len(v), 10, replace=False)
    for i in idx:
        e[:] = 0
        e[i] = 1.0
        assert abs((np.sum(Y * oracle.spmm(pat, v + e, X)) - f0) - g[i]) < 1e-10


# ----------------------------------------------------------------------------
# Chebyshev recurrence (kernel polynomial method, Sec. V)


def _diag_pattern(d):
    n = len(d)
    return BlockPattern(np.ones(n), np.ones(n), np.arange(n + 1), np.arange(n)), np.asarray(d, float)


def test_chebyshev_diagonal_closed_form():
    """H~ diagonal: with +-1 vectors t_n = T_n(H~) R exactly, so
    mu_n = (1/N) sum_p T_n(h_pp) = (1/N) sum_p cos(n arccos h_pp)."""
    h = np.linspace(-0.95, 0.9, 37)
    pat, v = _diag_pattern(h)
    R = syn.rademacher_panel(37, 4, 0)
    mu = oracle.chebyshev_moments(pat, v, R, 20)
    ref = np.array([np.mean(np.cos(n * np.arccos(h))) for n in range(20)])
    assert np.abs(mu - ref).max() < 1e-13


def test_chebyshev_zero_operator():
    """H~ = 0: T_n(0) = cos(n pi / 2) = 1, 0, -1, 0, ..."""
    pat, v = _diag_pattern(np.zeros(10))
    R = syn.rademacher_panel(10, 3, 1)
    mu = oracle.chebyshev_moments(pat, v, R, 12)
    exact = np.array([1.0, 0.0, -1.0, 0.0] * 3)
    assert np.array_equal(mu, exact)


def test_chebyshev_periodic_chain_exact_trace():
    """Periodic chain with hopping -1: eigenvalues -2 cos(2 pi m / N). With
    d = 2.02, c = 0 and R = sqrt(N) * identity (unit vectors scaled to the
    norm of a +-1 vector) the moments are the exact normalised traces
    (1/N) sum_m T_n(lambda_m / d)."""
    N = 24
    ptr = np.arange(0, 3 * N + 1, 3)
    cols = np.concatenate([sorted([(i - 1) % N, i, (i + 1) % N]) for i in range(N)])
    pat = BlockPattern(np.ones(N), np.ones(N), ptr, cols)
    v = np.array([0.0 if c == i else -1.0 for i in range(N) for c in sorted([(i - 1) % N, i, (i + 1) % N])])
    lam = -2 * np.cos(2 * np.pi * np.arange(N) / N)
    lo, hi = oracle.gershgorin_bounds(pat, v)
    assert lo <= lam.min() + 1e-12 and hi >= lam.max() - 1e-12
    c, d = 0.0, 2.02
    vt = oracle.shift_scale_values(pat, v, c, d)
    mu = oracle.chebyshev_moments(pat, vt, np.sqrt(N) * np.eye(N), 30)
    ref = np.array([np.mean(np.cos(n * np.arccos(lam / d))) for n in range(30)])
    assert np.abs(mu - ref).max() < 1e-13


def test_chebyshev_scaled_spectrum_and_bounded_moments():
    w = syn.tiny_multispecies(0)
    c, d = oracle.cheb_scale(w.pattern, w.values)
    vt = oracle.shift_scale_values(w.pattern, w.values, c, d)
    ev = np.linalg.eigvalsh(oracle.to_dense(w.pattern, vt))
    assert ev.min() > -1.0 and ev.max() < 1.0
    R = syn.rademacher_panel(w.pattern.n_rows, 4, 0)
    mu = oracle.chebyshev_moments(w.pattern, vt, R, 30)
    assert abs(mu[0] - 1.0) < 1e-15
    assert np.all(np.abs(mu) <= 1.0 + 1e-12)
    # the moments equal the dense-polynomial traces of the same random vectors
    Ht = oracle.to_dense(w.pattern, vt)
    T0, T1 = R, Ht @ R
    ref = [np.sum(R * T0) / R.size, np.sum(R * T1) / R.size]
    for n in range(2, 30):
        T0, T1 = T1, 2 * Ht @ T1 - T0
        ref.append(np.sum(R * T1) / R.size)
    assert np.abs(mu - np.array(ref)).max() < 1e-12


def test_moment_loss_gradient_central_differences():
    pat = syn.random_pattern(9, 9, (1, 2, 4), 0.35, 11)
    # square, with diagonal blocks only where sizes match
    pat = BlockPattern(pat.row_bsize, pat.row_bsize, pat.block_row_ptr, pat.block_col_idx)
    v = 0.3 * syn.random_values(pat, 11)
    R = syn.rademacher_panel(pat.n_rows, 3, 2)
    M = 8
    g = oracle.moment_loss_grad(pat, v, R, M)
    h = 1e-6
    rng = np.random.default_rng(0)
    for i in rng.choice(len(v), 20, replace=False):
        vp, vm = v.copy(), v.copy()
        vp[i] += h
        vm[i] -= h
        fd = (oracle.moment_loss(pat, vp, R, M) - oracle.moment_loss(pat, vm, R, M)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i]))


def test_gershgorin_matches_dense_definition():
    """Bounds from the dense matrix: min/max of H_rr -/+ sum_{c != r} |H_rc|."""
    pat = syn.random_pattern(15, 15, (1, 3, 4), 0.3, 31)
    pat = BlockPattern(pat.row_bsize, pat.row_bsize, pat.block_row_ptr, pat.block_col_idx)
    v = syn.random_values(pat, 31)
    H = oracle.to_dense(pat, v)
    d = np.diag(H)
    rad = np.abs(H).sum(axis=1) - np.abs(d)
    lo, hi = oracle.gershgorin_bounds(pat, v)
    assert abs(lo - (d - rad).min()) < 1e-13 and abs(hi - (d + rad).max()) < 1e-13


def test_kpm_doubling_moments_equal_direct_recurrence():
    """T_{2n} = 2 T_n^2 - 1 and T_{2n+1} = 2 T_{n+1} T_n - T_1 for a symmetric H."""
    w = syn.tiny_multispecies(0)
    c, d = oracle.cheb_scale(w.pattern, w.values)
    vt = oracle.shift_scale_values(w.pattern, w.values, c, d)
    R = syn.rademacher_panel(w.pattern.n_rows, 4, 2)
    for M in (1, 2, 3, 10, 31):
        a = oracle.kpm_moments_doubling(w.pattern, vt, R, M)
        b = oracle.chebyshev_moments(w.pattern, vt, R, M)
        assert np.abs(a - b).max() < 1e-13


def test_jackson_kernel_and_dos_normalisation():
    M = 64
    g = oracle.jackson_kernel(M)
    assert abs(g[0] - 1.0) < 1e-15 and np.all(np.diff(g) < 0) and g[-1] > 0
    # Chebyshev-Gauss quadrature on J > M nodes integrates rho exactly: integral = g_0 mu_0
    J = 4 * M
    xj = np.cos(np.pi * (np.arange(J) + 0.5) / J)
    mu = np.random.default_rng(0).uniform(-1, 1, M)
    mu[0] = 1.0
    rho = oracle.kpm_dos(mu, xj)
    integral = np.sum(rho * np.pi * np.sqrt(1 - xj ** 2)) / J
    assert abs(integral - 1.0) < 1e-13


def test_jackson_damped_delta_is_positive_and_localised():
    """The Jackson-damped expansion of a delta at x0 (mu_n = T_n(x0)) is
    non-negative and concentrated within a few pi/M of x0."""
    M, x0 = 128, 0.3
    mu = np.cos(np.arange(M) * np.arccos(x0))
    x = np.linspace(-0.999, 0.999, 4001)
    rho = oracle.kpm_dos(mu, x)
    assert rho.min() > -1e-12
    w = np.abs(x - x0) < 6 * np.pi / M
    dx = x[1] - x[0]
    assert np.sum(rho[w]) * dx > 0.99


def test_kpm_dos_of_diagonal_operator_counts_eigenvalues():
    """DOS of a diagonal H~ with exact traces (R = sqrt(N) I) integrates to the
    fraction of eigenvalues inside an interval (within the kernel's width)."""
    h = np.concatenate([np.full(30, -0.5), np.full(10, 0.4)])
    n = len(h)
    pat = BlockPattern(np.ones(n), np.ones(n), np.arange(n + 1), np.arange(n))
    mu = oracle.kpm_moments_doubling(pat, h, np.sqrt(n) * np.eye(n), 200)
    x = np.linspace(-0.999, 0.999, 8001)
    rho = oracle.kpm_dos(mu, x)
    dx = x[1] - x[0]
    assert abs(np.sum(rho[x < 0]) * dx - 0.75) < 1e-3
    assert abs(np.sum(rho[x > 0]) * dx - 0.25) < 1e-3


def test_central_difference_helper_against_plain_differences():
    """The cancellation-free central difference (tests/_fd.py) equals the
    plain (L+ - L-) / 2h at a step where the plain one is accurate."""
    from _fd import central_difference
    pat = syn.random_pattern(9, 9, (1, 2, 4), 0.35, 11)
    pat = syn.BlockPattern(pat.row_bsize, pat.row_bsize, pat.block_row_ptr, pat.block_col_idx)
    v = 0.3 * syn.random_values(pat, 11)
    R = syn.rademacher_panel(pat.n_rows, 3, 2)
    for i in (0, 7, len(v) - 1):
        h = 1e-3
        vp, vm = v.copy(), v.copy()
        vp[i] += h
        vm[i] -= h
        plain = (oracle.moment_loss(pat, vp, R, 8) - oracle.moment_loss(pat, vm, R, 8)) / (2 * h)
        assert abs(central_difference(pat, v, R, 8, i, h) - plain) <= 1e-9 * max(1.0, abs(plain))




def test_spgemm_eps0_is_dense_product():
    """With eps = 0 every block reached by a product path is kept and C = A B."""
    pa = syn.random_pattern(12, 9, (1, 3, 4), 0.3, 41)
    pb = syn.random_pattern(9, 11, (2, 5), 0.3, 42)
    pb = BlockPattern(pa.col_bsize, pb.col_bsize, pb.block_row_ptr, pb.block_col_idx)
    va, vb = syn.random_values(pa, 41), syn.random_values(pb, 42)
    rb, cb, ptr, cols, vals = oracle.spgemm(pa, va, pb, vb, 0.0)
    C = oracle.to_dense(BlockPattern(rb, cb, ptr, cols), vals)
    ref = oracle.to_dense(pa, va) @ oracle.to_dense(pb, vb)
    assert np.abs(C - ref).max() < 1e-13
    # every structurally reachable block is present, none else
    A0, B0 = oracle.to_dense(pa, np.ones(pa.nnz)), oracle.to_dense(pb, np.ones(pb.nnz))
    reach = (A0 @ B0) > 0
    present = oracle.to_dense(BlockPattern(rb, cb, ptr, cols), np.ones(len(vals))) > 0
    assert np.array_equal(reach, present)


def test_spgemm_threshold_respects_norm_bound():
    """Dropped blocks have true norm below eps (the Eq. 3 bound makes the
    symbolic drop safe); kept blocks equal the exact product blocks."""
    pa = syn.random_pattern(15, 15, (2, 3), 0.3, 43)
    pa = BlockPattern(pa.row_bsize, pa.row_bsize, pa.block_row_ptr, pa.block_col_idx)
    va = syn.random_values(pa, 43) * np.exp(-np.random.default_rng(0).uniform(0, 6, pa.nnz))
    exact = oracle.to_dense(pa, va) @ oracle.to_dense(pa, va)
    r = np.concatenate([[0], np.cumsum(pa.row_bsize)])
    eps = 0.5
    rb, cb, ptr, cols, vals = oracle.spgemm(pa, va, pa, va, eps)
    C = oracle.to_dense(BlockPattern(rb, cb, ptr, cols), vals)
    kept = set()
    for i in range(len(rb)):
        for u in range(ptr[i], ptr[i + 1]):
            kept.add((i, int(cols[u])))
    for i in range(len(rb)):
        for j in range(len(rb)):
            blk = exact[r[i]:r[i + 1], r[j]:r[j + 1]]
            if (i, j) in kept:
                assert np.allclose(C[r[i]:r[i + 1], r[j]:r[j + 1]], blk, atol=1e-13)
                assert np.linalg.norm(blk) >= eps - 1e-12
            else:
                assert np.linalg.norm(blk) < eps + 1e-12


# ----------------------------------------------------------------------------
# reciprocal-space sampling (Eq. 4) and complex block products


def test_kspace_chain_closed_form():
    """One orbital per cell, on-site e and hopping t to the neighbouring cells:
    the tight-binding band O(k) = e + 2 t cos(2 pi k_x)."""
    e, t = 0.3, -1.1
    ei, ej = [0, 0, 0], [0, 0, 0]
    eR = [0, 0, 0, 1, 0, 0, -1, 0, 0]
    vals = [e, t, t]
    for kx in (0.0, 0.1, 0.25, 0.5, 0.77):
        k = [kx, 0.3, -0.2]
        want = e + 2.0 * t * np.cos(2.0 * np.pi * kx)
        assert abs(oracle.kspace_dense([1], ei, ej, eR, vals, k)[0, 0] - want) < 1e-14
        *_, v = oracle.kspace_blocks([1], ei, ej, eR, vals, k)
        assert abs(v[0] - want) < 1e-14
    # the sign of Eq. 4: a lone forward hop (0, 0, R = +x) samples to t exp(-2 pi i k_x)
    H = oracle.kspace_dense([1], [0], [0], [1, 0, 0], [t], [0.25, 0, 0])
    assert abs(H[0, 0] - (-1j * t)) < 1e-15


def test_kspace_two_site_chain_band():
    """Two sites per cell, intra-cell hopping v and inter-cell hopping w: the
    bands are +-|v + w exp(2 pi i k)| (the dimerised chain), and the R+tau
    convention with tau = (0, 1/2) gives the same spectrum."""
    v, w = 0.7, 1.3
    ei, ej = [0, 1, 1, 0], [1, 0, 0, 1]
    eR = [0, 0, 0, 0, 0, 0, 1, 0, 0, -1, 0, 0]
    vals = [v, v, w, w]
    tau = [[0, 0, 0], [0.5, 0, 0]]
    for kx in (0.0, 0.13, 0.5, 0.81):
        band = abs(v + w * np.exp(2j * np.pi * kx))
        for tp in (None, tau):
            H = oracle.kspace_dense([1, 1], ei, ej, eR, vals, [kx, 0, 0], tp)
            assert np.allclose(H, H.conj().T, atol=1e-15)
            assert np.allclose(np.linalg.eigvalsh(H), [-band, band], atol=1e-14)


def _supercell_x2(w):
    """The same crystal as a 2 x 1 x 1 supercell: atom (i, m) = i + n m, edge
    (i, j, R) from cell m reaches cell m + R_x = 2 q + m' (m' in {0, 1})."""
    n = len(w.bsize)
    bi, bj, bR, bv = [], [], [], []
    off = np.concatenate([[0], np.cumsum(w.bsize[w.edge_i] * w.bsize[w.edge_j])])
    for m in (0, 1):
        for e in range(len(w.edge_i)):
            t = m + int(w.edge_R[e, 0])
            q, mp = t // 2, t % 2
            bi.append(int(w.edge_i[e]) + n * m)
            bj.append(int(w.edge_j[e]) + n * mp)
            bR.append([q, int(w.edge_R[e, 1]), int(w.edge_R[e, 2])])
            bv.append(w.edge_values[off[e]:off[e + 1]])
    return np.concatenate([w.bsize, w.bsize]), bi, bj, np.array(bR).ravel(), np.concatenate(bv)


def test_kspace_bloch_supercell_spectrum():
    """Bloch's theorem: the supercell operator doubled along x, sampled at
    K = (0, Ky, Kz), has the spectrum of O(k) at k = (0, Ky, Kz) and
    (1/2, Ky, Kz) together (zinc-blende cell with several images per pair)."""
    w = syn.zincblende_crystal(1)
    bs2, bi, bj, bR, bv = _supercell_x2(w)
    for ky, kz in ((0.0, 0.0), (0.21, -0.37)):
        Hs = oracle.kspace_dense(bs2, bi, bj, bR, bv, [0.0, ky, kz])
        e_super = np.linalg.eigvalsh(Hs)
        e_cell = np.concatenate([
            np.linalg.eigvalsh(oracle.kspace_dense(w.bsize, w.edge_i, w.edge_j, w.edge_R, w.edge_values,
                                                   [kx, ky, kz])) for kx in (0.0, 0.5)])
        assert np.allclose(np.sort(e_cell), e_super, atol=1e-11 * np.abs(e_super).max())


def test_kspace_invariants():
    """O(k + G) = O(k) for an integer G (R convention), O(k) Hermitian for the
    symmetric images, the R+tau convention equal to D O(k) D^dagger with
    D = diag(exp(2 pi i k . tau_i)), and the union-pattern blocks equal to the
    dense assembly."""
    w = syn.zincblende_crystal(1)
    args = (w.bsize, w.edge_i, w.edge_j, w.edge_R, w.edge_values)
    k = np.array([0.12, -0.31, 0.4])
    H = oracle.kspace_dense(*args, k)
    assert np.allclose(H, oracle.kspace_dense(*args, k + np.array([1, -2, 3])), atol=1e-12)
    assert np.allclose(H, H.conj().T, atol=1e-14)
    d = np.repeat(np.exp(2j * np.pi * (w.tau @ k)), w.bsize)
    Ht = oracle.kspace_dense(*args, k, w.tau)
    assert np.allclose(Ht, d[:, None] * H * d.conj()[None, :], atol=1e-13)
    rb, cb, ptr, cols, vals = oracle.kspace_blocks(*args, k)
    pat = BlockPattern(rb, cb, ptr, cols)
    assert np.allclose(oracle.to_dense(pat, vals.real) + 1j * oracle.to_dense(pat, vals.imag), H, atol=1e-14)


def test_complex_block_products_against_dense():
    """spmm_complex / spmm_adjoint_complex against dense complex algebra, the
    adjoint with the conjugate transpose, and <Y, H X> = <H^dagger Y, X>."""
    pat = syn.random_pattern(23, 19, (1, 3, 5, 8), 0.3, 61, empty_rows=2, unsorted=True)
    rng = np.random.default_rng(61)
    vals = rng.standard_normal(pat.nnz) + 1j * rng.standard_normal(pat.nnz)
    D = oracle.to_dense(pat, vals.real) + 1j * oracle.to_dense(pat, vals.imag)
    X = rng.standard_normal((pat.n_cols, 4)) + 1j * rng.standard_normal((pat.n_cols, 4))
    Y0 = rng.standard_normal((pat.n_rows, 4)) + 1j * rng.standard_normal((pat.n_rows, 4))
    got = oracle.spmm_complex(pat, vals, X, 2.0, -0.5, Y0)
    assert np.allclose(got, 2.0 * D @ X - 0.5 * Y0, atol=1e-13)
    Xa = rng.standard_normal((pat.n_rows, 3)) + 1j * rng.standard_normal((pat.n_rows, 3))
    ga = oracle.spmm_adjoint_complex(pat, vals, Xa)
    assert np.allclose(ga, D.conj().T @ Xa, atol=1e-13)
    Yv, Xv = Xa[:, :1], X[:, :1]
    lhs = np.vdot(Yv, oracle.spmm_complex(pat, vals, Xv))
    rhs = np.vdot(oracle.spmm_adjoint_complex(pat, vals, Yv), Xv)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_complex_chebyshev_moments_and_gershgorin():
    """For a Hermitian O(k): the Gershgorin interval holds the spectrum; the
    scaled moments equal sum_i |<v_i, R>|^2 T_n(lambda_i) / (N k) from a dense
    eigendecomposition (T_n(x) = cos(n arccos x)); at k = 0 with real vectors
    they equal the real recurrence's moments."""
    w = syn.zincblende_crystal(1)
    args = (w.bsize, w.edge_i, w.edge_j, w.edge_R, w.edge_values)
    rb, cb, ptr, cols, vals = oracle.kspace_blocks(*args, [0.21, -0.13, 0.34])
    pat = BlockPattern(rb, cb, ptr, cols)
    lo, hi = oracle.gershgorin_bounds_complex(pat, vals)
    D = oracle.to_dense(pat, vals.real) + 1j * oracle.to_dense(pat, vals.imag)
    ev = np.linalg.eigvalsh(D)
    assert lo <= ev.min() and ev.max() <= hi
    c, d = 0.5 * (hi + lo), 1.01 * 0.5 * (hi - lo)
    vt = oracle.shift_scale_values_complex(pat, vals, c, d)
    Dt = oracle.to_dense(pat, vt.real) + 1j * oracle.to_dense(pat, vt.imag)
    assert np.allclose(Dt, (D - c * np.eye(len(D))) / d, atol=1e-15)
    lam, V = np.linalg.eigh(Dt)
    rng = np.random.default_rng(0)
    R = np.exp(2j * np.pi * rng.random((len(D), 3)))          # random phases
    mu = oracle.chebyshev_moments_complex(pat, vt, R, 12)
    w2 = np.abs(V.conj().T @ R) ** 2                           # |<v_i, R_c>|^2
    th = np.arccos(np.clip(lam, -1, 1))
    ref = np.array([np.sum(w2 * np.cos(n * th)[:, None]) for n in range(12)]) / R.size
    assert np.allclose(mu, ref, atol=1e-12)
    # k = 0 sums real images: the complex recurrence with real vectors is the real one
    rb0, cb0, ptr0, cols0, v0 = oracle.kspace_blocks(*args, [0.0, 0.0, 0.0])
    p0 = BlockPattern(rb0, cb0, ptr0, cols0)
    assert np.abs(v0.imag).max() == 0.0
    assert np.allclose(oracle.gershgorin_bounds_complex(p0, v0), oracle.gershgorin_bounds(p0, v0.real), atol=1e-12)
    Rr = rng.choice([-1.0, 1.0], size=(len(D), 2))
    c0, d0 = oracle.cheb_scale(p0, v0.real)
    vt0 = oracle.shift_scale_values(p0, v0.real, c0, d0)
    assert np.allclose(oracle.chebyshev_moments_complex(p0, vt0.astype(np.complex128), Rr, 10),
                       oracle.chebyshev_moments(p0, vt0, Rr, 10), atol=1e-13)


def test_complex_gershgorin_matches_dense_definition():
    """Complex Hermitian O(k) at k != 0: the bounds are min / max over scalar
    rows of Re O_rr -/+ sum_{c != r} |O_rc|, computed here from the dense
    matrix (a modulus / real-part mix-up or a dropped imaginary part fails)."""
    w = syn.zincblende_crystal(1)
    for kf in ([0.21, -0.13, 0.34], [0.37, 0.12, 0.05], [0.07, 0.41, -0.29]):
        rb, cb, ptr, cols, vals = oracle.kspace_blocks(w.bsize, w.edge_i, w.edge_j, w.edge_R, w.edge_values, kf)
        pat = BlockPattern(rb, cb, ptr, cols)
        D = oracle.to_dense(pat, vals.real) + 1j * oracle.to_dense(pat, vals.imag)
        assert np.abs(D.imag).max() > 0.1            # a genuinely complex operator
        d = np.diag(D).real
        rad = np.abs(D).sum(axis=1) - np.abs(np.diag(D))
        lo, hi = oracle.gershgorin_bounds_complex(pat, vals)
        assert abs(lo - (d - rad).min()) <= 1e-13 * abs(lo)
        assert abs(hi - (d + rad).max()) <= 1e-13 * abs(hi)
        # the real-part-only radius (a plausible mistake) gives different bounds
        rad_re = np.abs(D.real).sum(axis=1) - np.abs(np.diag(D.real))
        assert abs(hi - (d + rad_re).max()) > 1e-6


def test_kpm_gap_on_a_step_density():
    """DOS 1 outside |E| < 0.3 and 0 inside, on a 401-point grid: the gap
    around 0 is the run of grid points with |E| < 0.3 (indices 141 .. 259),
    None inside a band, and a run that reaches the grid's end stops there."""
    E = np.linspace(-1.0, 1.0, 401)
    j = np.arange(401)
    D = np.where((j > 140) & (j < 260), 0.0, 1.0)
    assert oracle.kpm_gap(E, D, 0.0, 0.5) == (E[141], E[259])
    assert oracle.kpm_gap(E, D, 0.29, 0.5) == (E[141], E[259])
    assert oracle.kpm_gap(E, D, 0.6, 0.5) is None
    # the nearest grid point decides: a reference between two points, ties to the lower index
    assert oracle.kpm_gap(E, D, 0.5 * (E[259] + E[260]), 0.5) == (E[141], E[259])
    D2 = np.where(j > 350, 0.0, 1.0)
    assert oracle.kpm_gap(E, D2, 0.9, 0.5) == (E[351], E[400])
    # NaN is not below the threshold
    D3 = D.copy()
    D3[150] = np.nan
    assert oracle.kpm_gap(E, D3, 0.0, 0.5) == (E[151], E[259])


def test_kpm_gap_of_a_gapped_spectrum():
    """The whole DOS pipeline on a diagonal operator with eigenvalues filling
    [-0.9, -0.4] and [0.4, 0.9] (exact traces): the Jackson-damped DOS leaks
    into the gap by a few kernel widths pi / M, so the gap read at 2 % of the
    DOS maximum lies inside (-0.4, 0.4) and within 6 pi / M of its edges."""
    h = np.concatenate([np.linspace(-0.9, -0.4, 300), np.linspace(0.4, 0.9, 300)])
    n = len(h)
    pat = BlockPattern(np.ones(n), np.ones(n), np.arange(n + 1), np.arange(n))
    M = 256
    mu = oracle.kpm_moments_doubling(pat, h, np.sqrt(n) * np.eye(n), M)
    x = np.linspace(-0.999, 0.999, 2001)
    rho = oracle.kpm_dos(mu, x)
    lo, hi = oracle.kpm_gap(x, rho, 0.0, 0.02 * rho.max())
    assert -0.4 < lo < -0.4 + 6 * np.pi / M
    assert 0.4 - 6 * np.pi / M < hi < 0.4

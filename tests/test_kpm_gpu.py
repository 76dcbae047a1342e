"""GPU parity of the kernel-polynomial DOS pipeline: moments by the doubling
identities, Jackson-damped DOS reconstruction, gap helper."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


def _scaled(w):
    from paper_2609_04397_gb300 import VBCSR
    c, d = oracle.cheb_scale(w.pattern, w.values)
    vt = oracle.shift_scale_values(w.pattern, w.values, c, d)
    return VBCSR.from_pattern(w.pattern, vt, torch.float64, "cuda:0"), vt


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5, 30, 51])
def test_doubling_moments_match_oracle_and_direct(M):
    w = syn.tiny_multispecies(0)
    H, vt = _scaled(w)
    R = syn.rademacher_panel(w.pattern.n_rows, 8, 1)
    Rd = torch.from_numpy(R).cuda()
    got = H.kpm_moments(Rd, M).cpu().numpy()
    ref = oracle.kpm_moments_doubling(w.pattern, vt, R, M)
    assert np.abs(got - ref).max() <= 1e-12
    direct, _ = H.chebyshev(Rd, M)
    assert np.abs(got - direct.cpu().numpy()).max() <= 1e-12


@pytest.mark.parametrize("mode", ["tf32x3", "bf16x2", "df32"])
def test_doubling_moments_mixed_precision(mode):
    w = syn.amorphous(n=1500, side=60.0 * (1500 / 20000) ** (1 / 3), seed=2)
    H, vt = _scaled(w)
    R = syn.rademacher_panel(w.pattern.n_rows, 8, 0)
    got = H.kpm_moments(torch.from_numpy(R).cuda(), 64, precision=mode).cpu().numpy()
    ref = oracle.kpm_moments_doubling(w.pattern, vt, R, 64)
    tol = 1e-12 if mode == "df32" else 1e-5
    assert np.abs(got - ref).max() <= tol


@pytest.mark.parametrize("kernel", ["jackson", "none"])
def test_dos_reconstruction_matches_oracle(kernel):
    from paper_2609_04397_gb300 import kpm_dos
    rng = np.random.default_rng(5)
    for M in (1, 7, 300, 2500):
        mu = rng.uniform(-1, 1, M) / np.sqrt(1 + np.arange(M))
        mu[0] = 1.0
        x = np.linspace(-0.995, 0.995, 1001)
        got = kpm_dos(torch.from_numpy(mu).cuda(), torch.from_numpy(x).cuda(), kernel).cpu().numpy()
        ref = oracle.kpm_dos(mu, x, kernel)
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_dos_pipeline_and_gap_on_a_gapped_operator():
    """Diagonal operator with eigenvalues in two bands [-0.8, -0.2] and
    [0.3, 0.9]: the reconstructed DOS integrates to the band fractions and the
    gap helper finds the empty interval between them."""
    from paper_2609_04397_gb300 import VBCSR, kpm_dos, kpm_gap
    n = 600
    h = np.concatenate([np.linspace(-0.8, -0.2, 400), np.linspace(0.3, 0.9, 200)])
    pat = syn.BlockPattern(np.ones(n, np.int32), np.ones(n, np.int32), np.arange(n + 1), np.arange(n))
    H = VBCSR.from_pattern(pat, h, torch.float64, "cuda:0")
    R = torch.from_numpy(syn.rademacher_panel(n, 32, 0)).cuda()
    mu = H.kpm_moments(R, 256)
    x = torch.linspace(-0.999, 0.999, 4001, dtype=torch.float64, device="cuda:0")
    rho = kpm_dos(mu, x).cpu().numpy()
    xs = x.cpu().numpy()
    dx = xs[1] - xs[0]
    assert abs(np.sum(rho[xs < 0.05]) * dx - 400 / 600) < 2e-2
    thr = 0.05 * rho.max()
    lo, hi = kpm_gap(x, torch.from_numpy(rho).cuda(), 0.05, thr)
    assert -0.2 < lo < 0.0 and 0.1 < hi < 0.3
    assert (lo, hi) == oracle.kpm_gap(xs, rho, 0.05, thr)


def test_gap_search_matches_oracle_exactly():
    """vbcsr_kpm_gap against the oracle's walk on many random grids: the same
    two grid energies (or none), bit for bit, including ties of the nearest
    grid point, NaN densities, runs that reach the grid's ends, references
    outside the grid and grids longer than the CTA."""
    from paper_2609_04397_gb300 import kpm_gap
    rng = np.random.default_rng(3)
    for trial in range(60):
        n = int(rng.choice([1, 2, 7, 64, 1023, 1024, 1025, 5000]))
        E = np.sort(rng.uniform(-1, 1, n)) if trial % 3 else np.linspace(-1, 1, n)
        D = rng.uniform(0, 1, n) ** 3
        if trial % 5 == 0:
            D[rng.integers(0, n, max(1, n // 50))] = np.nan
        ref = float(rng.uniform(-1.2, 1.2)) if trial % 7 else float(0.5 * (E[0] + E[-1]))
        thr = float(rng.uniform(0.05, 0.6))
        got = kpm_gap(torch.from_numpy(E).cuda(), torch.from_numpy(D).cuda(), ref, thr)
        assert got == oracle.kpm_gap(E, D, ref, thr), (trial, n, ref, thr)

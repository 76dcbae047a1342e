"""GPU parity of the Chebyshev recurrence (kernel polynomial method, Sec. V),
its checkpoints, its mixed-precision form and its reverse-mode gradient."""
import os

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn
from _fd import central_difference

pytestmark = pytest.mark.gpu


def _setup(w):
    from paper_2609_04397_gb300 import VBCSR
    c, d = oracle.cheb_scale(w.pattern, w.values)
    vt = oracle.shift_scale_values(w.pattern, w.values, c, d)
    H = VBCSR.from_pattern(w.pattern, vt, torch.float64, "cuda:0")
    return H, vt, c, d


def test_moments_and_checkpoints_tiny():
    w = syn.tiny_multispecies(0)
    H, vt, c, d = _setup(w)
    R = syn.rademacher_panel(w.pattern.n_rows, 16, 0)
    M, E = 30, 10
    mom, ck = H.chebyshev(torch.from_numpy(R).cuda(), M, ckpt_every=E)
    ref = oracle.chebyshev_moments(w.pattern, vt, R, M)
    assert np.abs(mom.cpu().numpy() - ref).max() <= 1e-12
    t = oracle.chebyshev_vectors(w.pattern, vt, R, M)
    ck = ck.cpu().numpy()
    assert ck.shape[0] == 3
    for s in range(ck.shape[0]):
        for j in range(2):
            ref_t = t[s * E + j]
            assert np.linalg.norm(ck[s, j] - ref_t) <= 1e-12 * np.linalg.norm(ref_t)


@pytest.mark.parametrize("mode", ["f32", "tf32x3", "bf16x2"])
def test_mixed_precision_moments(mode):
    """Block products in reduced precision, recurrence and moments in FP64:
    every moment within 1e-5 of the FP64 oracle (relative to mu_0 = 1)."""
    w = syn.tiny_multispecies(0)
    H, vt, c, d = _setup(w)
    R = syn.rademacher_panel(w.pattern.n_rows, 16, 0)
    mom, _ = H.chebyshev(torch.from_numpy(R).cuda(), 51, precision=mode)
    ref = oracle.chebyshev_moments(w.pattern, vt, R, 51)
    err = np.abs(mom.cpu().numpy() - ref) / abs(ref[0])
    assert err.max() <= 1e-5, err.max()


def test_df32_moments_fp64_accurate():
    """Double-FP32 block products inside the FP64 recurrence: moments within
    the FP64 moment tolerance."""
    w = syn.tiny_multispecies(0)
    H, vt, c, d = _setup(w)
    R = syn.rademacher_panel(w.pattern.n_rows, 16, 0)
    mom, _ = H.chebyshev(torch.from_numpy(R).cuda(), 51, precision="df32")
    ref = oracle.chebyshev_moments(w.pattern, vt, R, 51)
    assert np.abs(mom.cpu().numpy() - ref).max() <= 1e-12


def _grad_case(n_atoms, k, M, E, seed=0):
    side = 60.0 * (n_atoms / 20000) ** (1 / 3)
    w = syn.amorphous(n=n_atoms, side=side, seed=seed)
    H, vt, c, d = _setup(w)
    R = syn.rademacher_panel(w.pattern.n_rows, k, seed)
    return w, H, vt, c, d, R


@pytest.mark.parametrize("E", [1, 4, 10, 40])
def test_moment_loss_gradient_matches_oracle(E):
    from paper_2609_04397_gb300 import chebyshev_moments
    w, H, vt, c, d, R = _grad_case(600, 4, 30, E)
    v = torch.from_numpy(vt).cuda().requires_grad_(True)
    mu = chebyshev_moments(H, v, torch.from_numpy(R).cuda(), 30, ckpt_every=E)
    loss = (mu ** 2).sum()
    loss.backward()
    ref = oracle.moment_loss_grad(w.pattern, vt, R, 30)
    g = v.grad.cpu().numpy()
    assert np.linalg.norm(g - ref) <= 1e-11 * np.linalg.norm(ref)
    assert np.abs(g - ref).max() <= 1e-10 * np.abs(ref).max()


def test_gradient_through_shift_scale_and_fd():
    """Moments of H~ = (H - c I) / d formed in the library from the values of
    H; dL/dH (original values) = dL/dH~ / d, also formed in the library,
    checked against the oracle's reverse-mode gradient and against central
    finite differences (h = 1e-6) of the oracle's loss on 50 sampled entries."""
    from paper_2609_04397_gb300 import chebyshev_moments
    w, H, vt, c, d, R = _grad_case(300, 4, 30, 10)
    v = torch.from_numpy(w.values).cuda().requires_grad_(True)
    mu = chebyshev_moments(H, v, torch.from_numpy(R).cuda(), 30, ckpt_every=10, c=c, d=d)
    ref_mu = oracle.chebyshev_moments(w.pattern, vt, R, 30)
    assert np.abs(mu.detach().cpu().numpy() - ref_mu).max() <= 1e-12
    (mu ** 2).sum().backward()
    g = v.grad.cpu().numpy()
    ref = oracle.moment_loss_grad(w.pattern, vt, R, 30) / d
    assert np.linalg.norm(g - ref) <= 1e-12 * np.linalg.norm(ref)

    h = 1e-6
    idx = np.random.default_rng(0).choice(len(vt), 50, replace=False)
    # dL/dH = dL/dH~ / d: the central difference in H~ at step h / d is the one in H at step h
    fd = np.array([central_difference(w.pattern, vt, R, 30, i, h / d) / d for i in idx])
    # max-norm relative deviation over the sampled entries
    assert np.abs(fd - g[idx]).max() <= 1e-6 * np.abs(g[idx]).max()


def test_f32_products_gradient_close_to_fp64():
    from paper_2609_04397_gb300 import chebyshev_moments
    w, H, vt, c, d, R = _grad_case(600, 4, 30, 10)
    Rd = torch.from_numpy(R).cuda()
    grads = {}
    for mode in ("native", "f32"):
        v = torch.from_numpy(vt).cuda().requires_grad_(True)
        (chebyshev_moments(H, v, Rd, 30, 10, precision=mode) ** 2).sum().backward()
        grads[mode] = v.grad.cpu().numpy()
    rel = np.linalg.norm(grads["f32"] - grads["native"]) / np.linalg.norm(grads["native"])
    assert rel <= 1e-4, rel


def test_matmul_autograd():
    from paper_2609_04397_gb300 import VBCSR, vbcsr_matmul
    pat = syn.random_pattern(30, 25, (4, 9, 13), 0.2, 2)
    vals = syn.random_values(pat, 2)
    H = VBCSR.from_pattern(pat, vals, torch.float64, "cuda:0")
    X = np.random.default_rng(1).standard_normal((pat.n_cols, 6))
    G = np.random.default_rng(2).standard_normal((pat.n_rows, 6))
    v = torch.from_numpy(vals).cuda().requires_grad_(True)
    Xd = torch.from_numpy(X).cuda().requires_grad_(True)
    Y = vbcsr_matmul(H, v, Xd)
    (Y * torch.from_numpy(G).cuda()).sum().backward()
    ref_dx = oracle.spmm_adjoint(pat, vals, G)
    ref_dv = oracle.sddmm(pat, G, X)
    assert np.linalg.norm(Xd.grad.cpu().numpy() - ref_dx) <= 1e-12 * np.linalg.norm(ref_dx)
    assert np.linalg.norm(v.grad.cpu().numpy() - ref_dv) <= 1e-12 * np.linalg.norm(ref_dv)


def test_amorphous_20k_gradient_fd_50_entries():
    """Full differentiation workload: 20k amorphous atoms, 30 moments, k = 16,
    checkpoints every 10 steps; GPU gradient of L = sum mu_n^2 against central
    differences (h = 1e-6) of the oracle on 50 sampled stored entries, against
    the oracle's exact reverse-mode gradient on every entry, and the gradient
    with FP32 block products against the FP64 one (within 1e-4)."""
    import time
    from paper_2609_04397_gb300 import chebyshev_moments
    w, H, vt, c, d, R = _grad_case(20000, 16, 30, 10)
    Rd = torch.from_numpy(R).cuda()
    grads = {}
    for mode in ("native", "f32"):
        v = torch.from_numpy(vt).cuda().requires_grad_(True)
        (chebyshev_moments(H, v, Rd, 30, ckpt_every=10, precision=mode) ** 2).sum().backward()
        grads[mode] = v.grad.cpu().numpy()
    g = grads["native"]
    rel32 = np.linalg.norm(grads["f32"] - g) / np.linalg.norm(g)
    assert rel32 <= 1e-4, rel32
    nthreads = os.cpu_count() or 1
    pat = w.pattern

    t0 = time.perf_counter()
    h = 1e-6
    idx = np.random.default_rng(0).choice(len(vt), 50, replace=False)
    fd = np.array([central_difference(pat, vt, R, 30, i, h, nthreads) for i in idx])
    worst = np.abs(fd - g[idx]).max() / np.abs(g[idx]).max()
    print(f"amorphous 20k: max-norm relative FD deviation over 50 entries = {worst:.3e} "
          f"({time.perf_counter() - t0:.0f} s of oracle time on {nthreads} threads); "
          f"FP32-product gradient vs FP64: {rel32:.2e}")
    assert worst <= 1e-6
    # and the exact reverse-mode gradient of the oracle, every stored entry
    ref = oracle.moment_loss_grad(pat, vt, R, 30)
    assert np.linalg.norm(g - ref) <= 1e-12 * np.linalg.norm(ref)


def test_gershgorin_and_shift_scale_on_gpu():
    from paper_2609_04397_gb300 import VBCSR
    w = syn.amorphous(n=500, side=60.0 * (500 / 20000) ** (1 / 3), seed=3)
    H = VBCSR.from_pattern(w.pattern, w.values, torch.float64, "cuda:0")
    lo, hi = H.gershgorin()
    rlo, rhi = oracle.gershgorin_bounds(w.pattern, w.values)
    assert abs(lo - rlo) <= 1e-13 * abs(rlo) and abs(hi - rhi) <= 1e-13 * abs(rhi)
    c, d = 0.5 * (hi + lo), 1.01 * 0.5 * (hi - lo)
    H.spmm(torch.ones(w.pattern.n_cols, 2, dtype=torch.float64, device="cuda:0"), precision="bf16x2")
    H.shift_scale(c, d)
    ref = oracle.shift_scale_values(w.pattern, w.values, c, d)
    assert np.array_equal(H.get_values().cpu().numpy(), ref)
    # the mixed-precision copy follows the new values
    X = np.random.default_rng(0).standard_normal((w.pattern.n_cols, 3))
    got = H.spmm(torch.from_numpy(X).cuda(), precision="bf16x2").cpu().numpy()
    refy = oracle.spmm(w.pattern, ref, X)
    assert np.linalg.norm(got - refy) <= 1e-5 * np.linalg.norm(refy)


def test_recurrence_captured_in_a_cuda_graph():
    """The whole Chebyshev recurrence (one product with fused epilogue and
    dot per step, the dot finalisation, the copies) is stream-ordered with no
    host synchronisation or allocation after a first call, so it can be
    captured once and replayed: a small system is launch-bound, and a replay
    pays one graph launch instead of ~3 per step. The replay gives the eager
    moments bit for bit and follows new vectors written into the captured R."""
    from paper_2609_04397_gb300 import lib
    import ctypes
    w = syn.tiny_multispecies(0)
    H, vt, c, d = _setup(w)
    N, k, M = w.pattern.n_rows, 4, 40
    R = torch.from_numpy(syn.rademacher_panel(N, k, 0)).cuda()
    mom = torch.empty(M, dtype=torch.float64, device="cuda:0")
    work = torch.empty(2 * N * k, dtype=torch.float64, device="cuda:0")

    def run():
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = lib().vbcsr_chebyshev(H._h, k, ctypes.c_void_p(R.data_ptr()), k, M, ctypes.c_void_p(mom.data_ptr()),
                                   ctypes.c_void_p(work.data_ptr()), None, 0, 0, st)
        assert rc == 0

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        run()                                   # first call outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager = mom.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run()
    mom.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(mom, eager)
    R2 = syn.rademacher_panel(N, k, 7)
    R.copy_(torch.from_numpy(R2))
    g.replay()
    torch.cuda.synchronize()
    ref = oracle.chebyshev_moments(w.pattern, vt, R2, M)
    assert np.abs(mom.cpu().numpy() - ref).max() <= 1e-12
    # timing of the launch-bound case, eager against replay (reported, not asserted)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        run()
    e1.record()
    torch.cuda.synchronize()
    t_eager = e0.elapsed_time(e1) / 20
    e0.record()
    for _ in range(20):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    print(f"tiny Chebyshev recurrence, {M} moments: eager {t_eager:.3f} ms, graph {e0.elapsed_time(e1) / 20:.3f} ms")

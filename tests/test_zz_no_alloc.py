"""The allocation-free Chebyshev entry point (vbcsr_chebyshev_noalloc).

It serves callers that cannot allocate device memory when they need the
moments (their memory belongs to another allocator that reserved it up front,
or their loop must not allocate): the work panels live in a fixed array inside
the library. Here it is called through the C ABI twice in a row, in every
precision, and must give the moments of the existing vbcsr_chebyshev (which
uses a caller-allocated work buffer) within the FP64 moment tolerance of the
other tests (1e-12 of mu_0); the second call must not change the device's free
memory. A mixed-precision mode runs only once an ordinary call has built the
handle's buffers for it; requests beyond the array (a complex panel counts two
doubles per element) are refused before anything is launched.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = 1e-12
PREC = {"native": 0, "f32": 1, "tf32": 2, "tf32x3": 3, "bf16x2": 4, "df32": 5}


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _moments_existing(L, H, R, M, prec=0):
    N, k = R.shape
    mom = torch.empty(M, dtype=torch.float64, device="cuda:0")
    work = torch.empty(2 * N * k, dtype=R.dtype, device="cuda:0")
    rc = L.vbcsr_chebyshev(H.handle, k, ctypes.c_void_p(R.data_ptr()), k, M, ctypes.c_void_p(mom.data_ptr()),
                           ctypes.c_void_p(work.data_ptr()), None, 0, prec, _stream())
    assert rc == 0, L.vbcsr_last_error_detail()
    return mom


def _moments_noalloc(L, H, R, M, mom, prec=0):
    N, k = R.shape
    return L.vbcsr_chebyshev_noalloc(H.handle, k, ctypes.c_void_p(R.data_ptr()), k, M,
                                     ctypes.c_void_p(mom.data_ptr()), prec, _stream())


def _scaled_tiny():
    from paper_2609_04397_gb300 import VBCSR
    w = syn.tiny_multispecies(0)
    c, d = oracle.cheb_scale(w.pattern, w.values)
    vt = oracle.shift_scale_values(w.pattern, w.values, c, d)
    return w, VBCSR.from_pattern(w.pattern, vt, torch.float64, "cuda:0")


@pytest.mark.parametrize("prec", list(PREC))
def test_noalloc_matches_existing_entry_point_twice(prec):
    from paper_2609_04397_gb300 import lib
    L = lib()
    w, H = _scaled_tiny()
    M = 30
    out = torch.empty(M, dtype=torch.float64, device="cuda:0")
    for call, seed in enumerate((0, 1)):
        R = torch.from_numpy(syn.rademacher_panel(w.pattern.n_rows, 16, seed)).cuda()
        # the ordinary call (first: it also builds the mode's buffers on the handle)
        ref = _moments_existing(L, H, R, M, PREC[prec])
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        out.fill_(float("nan"))
        rc = _moments_noalloc(L, H, R, M, out, PREC[prec])
        assert rc == 0, L.vbcsr_last_error_detail()
        torch.cuda.synchronize()
        if call == 1:       # after the first call's one-time set-up, nothing is allocated
            assert torch.cuda.mem_get_info()[0] == free_before
        err = (out - ref).abs().max().item() / abs(ref[0].item())
        assert err <= TOL, (prec, call, err)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x2", "df32"])
def test_noalloc_refuses_a_mode_whose_buffers_are_not_built(prec):
    from paper_2609_04397_gb300 import lib
    L = lib()
    w, H = _scaled_tiny()
    R = torch.from_numpy(syn.rademacher_panel(w.pattern.n_rows, 16, 0)).cuda()
    mom = torch.zeros(6, dtype=torch.float64, device="cuda:0")
    free_before = torch.cuda.mem_get_info()[0]
    assert _moments_noalloc(L, H, R, 6, mom, PREC[prec]) == -5
    assert b"has not built yet" in L.vbcsr_last_error_detail()
    torch.cuda.synchronize()
    assert torch.count_nonzero(mom).item() == 0       # nothing was launched
    assert torch.cuda.mem_get_info()[0] == free_before
    # buffers built for 8 columns are not enough for 16
    _moments_existing(L, H, R[:, :8].contiguous(), 6, PREC[prec])
    assert _moments_noalloc(L, H, R, 6, mom, PREC[prec]) == -5
    # once an ordinary call has built them for 16 columns, the call runs
    _moments_existing(L, H, R, 6, PREC[prec])
    assert _moments_noalloc(L, H, R, 6, mom, PREC[prec]) == 0


def test_noalloc_rejects_requests_beyond_its_work_area():
    from paper_2609_04397_gb300 import VBCSR, lib
    L = lib()
    n = 70_000                      # 70,000 rows x 16 > 2^20 elements per panel
    pat = syn.BlockPattern(np.ones(n, np.int32), np.ones(n, np.int32), np.arange(n + 1), np.arange(n))
    H = VBCSR.from_pattern(pat, np.full(n, 0.5), torch.float64, "cuda:0")
    R = torch.ones((n, 16), dtype=torch.float64, device="cuda:0")
    mom = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    rc = _moments_noalloc(L, H, R, 4, mom)
    assert rc == -5
    assert b"exceeds the fixed work area" in L.vbcsr_last_error_detail()
    torch.cuda.synchronize()
    assert torch.count_nonzero(mom).item() == 0       # nothing was launched


def test_noalloc_complex_panels_count_two_doubles_per_element():
    """A complex operator's panel element is two doubles: 40,000 rows x 16
    columns is under 2^20 elements but over 2^20 doubles, so it is refused;
    a small complex case runs and matches the existing entry point."""
    from paper_2609_04397_gb300 import VBCSR, lib
    L = lib()
    n = 40_000
    ei = np.arange(n, dtype=np.int32)
    H = VBCSR.from_images(np.ones(n, np.int32), ei, ei, np.zeros((n, 3), np.int32), np.full(n, 0.5),
                          device="cuda:0")
    H.set_kpoint([0.0, 0.0, 0.0])
    R = torch.ones((n, 16), dtype=torch.complex128, device="cuda:0")
    mom = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    assert _moments_noalloc(L, H, R, 4, mom) == -5
    assert b"(complex)" in L.vbcsr_last_error_detail()
    torch.cuda.synchronize()
    assert torch.count_nonzero(mom).item() == 0

    w = syn.zincblende_crystal(1)
    Hc = VBCSR.from_images(w.bsize, w.edge_i, w.edge_j, w.edge_R, w.edge_values, device="cuda:0")
    Hc.set_kpoint([0.1, 0.2, 0.3])
    lo, hi = Hc.gershgorin()
    Hc.shift_scale(0.5 * (hi + lo), 1.01 * 0.5 * (hi - lo))
    N = Hc.shape[0]
    rng = np.random.default_rng(0)
    Rc = torch.from_numpy(np.exp(2j * np.pi * rng.random((N, 4)))).to("cuda:0")
    ref = _moments_existing(L, Hc, Rc, 20)
    out = torch.empty(20, dtype=torch.float64, device="cuda:0")
    for _ in range(2):
        assert _moments_noalloc(L, Hc, Rc, 20, out) == 0, L.vbcsr_last_error_detail()
        torch.cuda.synchronize()
        assert (out - ref).abs().max().item() <= TOL * abs(ref[0].item())

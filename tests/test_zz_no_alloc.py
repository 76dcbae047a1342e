"""The allocation-free Chebyshev entry point (vbcsr_chebyshev_noalloc).

It serves callers that cannot allocate device memory when they need the
moments (their memory belongs to another allocator, or their loop must not
allocate): its work panels live in a fixed array inside the library. Here it
is called through the C ABI twice in a row and must give the moments of the
existing vbcsr_chebyshev, which uses a caller-allocated work buffer, within
the FP64 moment tolerance of the other tests (1e-12); it must not change the
device's free memory, and it must refuse a request larger than its array.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _moments_existing(L, H, R, M):
    N, k = R.shape
    mom = torch.empty(M, dtype=torch.float64, device="cuda:0")
    work = torch.empty(2 * N * k, dtype=torch.float64, device="cuda:0")
    rc = L.vbcsr_chebyshev(H.handle, k, ctypes.c_void_p(R.data_ptr()), k, M, ctypes.c_void_p(mom.data_ptr()),
                           ctypes.c_void_p(work.data_ptr()), None, 0, 0, _stream())
    assert rc == 0, L.vbcsr_last_error_detail()
    return mom


def _moments_noalloc(L, H, R, M, mom):
    N, k = R.shape
    return L.vbcsr_chebyshev_noalloc(H.handle, k, ctypes.c_void_p(R.data_ptr()), k, M,
                                     ctypes.c_void_p(mom.data_ptr()), 0, _stream())


def test_noalloc_matches_existing_entry_point_twice():
    from paper_2609_04397_gb300 import VBCSR, lib
    L = lib()
    w = syn.tiny_multispecies(0)
    c, d = oracle.cheb_scale(w.pattern, w.values)
    vt = oracle.shift_scale_values(w.pattern, w.values, c, d)
    H = VBCSR.from_pattern(w.pattern, vt, torch.float64, "cuda:0")
    M = 30
    out = torch.empty(M, dtype=torch.float64, device="cuda:0")
    for call, seed in enumerate((0, 1)):
        R = torch.from_numpy(syn.rademacher_panel(w.pattern.n_rows, 16, seed)).cuda()
        ref = _moments_existing(L, H, R, M)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        out.fill_(float("nan"))
        rc = _moments_noalloc(L, H, R, M, out)
        assert rc == 0, L.vbcsr_last_error_detail()
        torch.cuda.synchronize()
        if call == 1:       # after the first call's one-time set-up, nothing is allocated
            assert torch.cuda.mem_get_info()[0] == free_before
        err = (out - ref).abs().max().item() / abs(ref[0].item())
        assert err <= TOL, (call, err)


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
    assert torch.count_nonzero(mom).item() == 0       # nothing was launched

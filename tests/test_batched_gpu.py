"""One operator over many independent structures of uneven size: parity with
the per-structure oracle, the persistent one-launch schedule, the autotuner
and CUDA-graph replay."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as syn
from synthetic.structures import BlockPattern
from _parity import TOL_F64, TOL_MIXED, check_elementwise, forward_ref, rel_fro

pytestmark = pytest.mark.gpu


def _batched(n_structs=24, n_max=400, dtype=torch.float32, seed=1):
    from paper_2609_04397_gb300 import VBCSR
    w = syn.batched_uneven(n_structs=n_structs, n_min=50, n_max=n_max, seed=seed)
    pat = w.pattern
    offs = w.struct_brow_offsets
    # local column indices, as vbcsr_create_batched takes them
    rows = pat.block_rows()
    s_of_row = np.searchsorted(offs, rows, side="right") - 1
    local = pat.block_col_idx.astype(np.int64) - offs[s_of_row]
    vals = w.values.astype(np.float32) if dtype == torch.float32 else w.values
    H = VBCSR.from_batched(offs, offs, pat.row_bsize, pat.col_bsize, pat.block_row_ptr, local, vals, dtype, "cuda:0")
    return w, H, vals.astype(np.float64)


def _per_structure_ref(w, vals, X):
    """Every structure separately through the oracle, results stacked."""
    out = []
    voff = w.pattern.value_offset()
    coff = np.concatenate([[0], np.cumsum(w.pattern.col_bsize.astype(np.int64))])
    for s, part in enumerate(w.parts):
        b0, b1 = w.struct_brow_offsets[s], w.struct_brow_offsets[s + 1]
        v = vals[voff[w.pattern.block_row_ptr[b0]]:voff[w.pattern.block_row_ptr[b1]]]
        out.append(oracle.spmm(part, v, X[coff[b0]:coff[b1]]))
    return np.concatenate(out)


def test_batched_matches_per_structure_oracle():
    w, H, vals = _batched()
    assert H.info.n_structs == 24
    X = np.random.default_rng(0).standard_normal((w.pattern.n_cols, 8)).astype(np.float32).astype(np.float64)
    got = H.spmm(torch.from_numpy(X).float().cuda()).cpu().numpy().astype(np.float64)
    ref = _per_structure_ref(w, vals, X)
    ref2, scale = forward_ref(w.pattern, vals, X, 1.0, 0.0, None)
    assert np.array_equal(ref, ref2)          # block-diagonal operator == independent structures
    assert rel_fro(got, ref) <= TOL_MIXED
    check_elementwise(got, ref, scale, 1e-4)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_persistent_schedule_equals_bucketed(dtype):
    """The persistent launch runs the bucketed launches' per-item arithmetic
    (bit for bit); the pipelined FP32 kernel, which the persistent launch on
    FP32 values uses at k >= 8, sums each entry in another order and agrees to
    FP32 rounding."""
    w, H, vals = _batched(dtype=dtype)
    X = torch.randn(w.pattern.n_cols, 8, dtype=dtype, device="cuda:0")
    H.set_schedule("bucketed")
    Yb = H.spmm(X)
    for warps in (0, 2, 8):
        H.set_schedule("persistent", warps, pipelined_f32=False)
        Yp = H.spmm(X)
        assert torch.equal(Yb, Yp)     # same per-item arithmetic, only the launch differs
        Ya = H.spmm_adjoint(X)
        H.set_schedule("bucketed")
        assert torch.equal(Ya, H.spmm_adjoint(X))
    H.set_schedule("persistent")
    Yq = H.spmm(X)
    if dtype == torch.float64:
        assert torch.equal(Yb, Yq)
    else:
        _, scale = forward_ref(w.pattern, np.abs(vals), np.abs(X.double().cpu().numpy()), 1.0, 0.0, None)
        check_elementwise(Yq.double().cpu().numpy(), Yb.double().cpu().numpy(), scale, 1e-5)


@pytest.mark.parametrize("k", [1, 8, 20])
def test_autotuned_parity(k, tmp_path):
    w, H, vals = _batched(dtype=torch.float64)
    t = H.autotune(k, cache=str(tmp_path / "tune.json"))
    assert t["schedule"] in ("bucketed", "persistent")
    t2 = H.autotune(k, cache=str(tmp_path / "tune.json"))   # second call: cache hit
    assert t2 == t
    X = np.random.default_rng(k).standard_normal((w.pattern.n_cols, k))
    got = H.spmm(torch.from_numpy(X).cuda()).cpu().numpy()
    ref, scale = forward_ref(w.pattern, vals, X, 1.0, 0.0, None)
    assert rel_fro(got, ref) <= TOL_F64
    check_elementwise(got, ref, scale, TOL_F64)


def test_cuda_graph_replay_persistent():
    w, H, vals = _batched(dtype=torch.float64)
    H.set_schedule("persistent")
    X = torch.zeros(w.pattern.n_cols, 8, dtype=torch.float64, device="cuda:0")
    Y = torch.empty(w.pattern.n_rows, 8, dtype=torch.float64, device="cuda:0")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        H.spmm(X, 1.0, 0.0, Y)          # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        H.spmm(X, 1.0, 0.0, Y)
    for seed in (1, 2):
        Xh = np.random.default_rng(seed).standard_normal((w.pattern.n_cols, 8))
        X.copy_(torch.from_numpy(Xh))
        g.replay()
        torch.cuda.synchronize()
        ref, scale = forward_ref(w.pattern, vals, Xh, 1.0, 0.0, None)
        check_elementwise(Y.cpu().numpy(), ref, scale, TOL_F64)


def test_many_separate_handles_agree_with_batched():
    from paper_2609_04397_gb300 import VBCSR
    w, H, vals = _batched(n_structs=8, dtype=torch.float64)
    X = torch.randn(w.pattern.n_cols, 8, dtype=torch.float64, device="cuda:0")
    Y = H.spmm(X)
    voff = w.pattern.value_offset()
    coff = np.concatenate([[0], np.cumsum(w.pattern.col_bsize.astype(np.int64))])
    for s, part in enumerate(w.parts):
        b0, b1 = w.struct_brow_offsets[s], w.struct_brow_offsets[s + 1]
        v = vals[voff[w.pattern.block_row_ptr[b0]]:voff[w.pattern.block_row_ptr[b1]]]
        Hs = VBCSR.from_pattern(part, v, torch.float64, "cuda:0")
        Ys = Hs.spmm(X[coff[b0]:coff[b1]].contiguous())
        assert torch.equal(Ys, Y[coff[b0]:coff[b1]])


def test_batched_rejects_bad_local_columns():
    from paper_2609_04397_gb300 import VBCSR, VBCSRError
    pat = BlockPattern(np.array([2, 2]), np.array([2, 2]), np.array([0, 1, 2]), np.array([0, 1]))
    with pytest.raises(VBCSRError) as ei:
        # two structures of one block each: local column 1 is outside structure 1
        VBCSR.from_batched([0, 1, 2], [0, 1, 2], pat.row_bsize, pat.col_bsize, pat.block_row_ptr,
                           np.array([0, 1]), np.ones(8), torch.float64, "cuda:0")
    assert ei.value.status == -2


def test_schedule_flags_round_trip_and_validation():
    """Every schedule flag reads back through get_tuning and survives
    apply_tuning; an unknown bit or a bad CTA width is rejected."""
    from paper_2609_04397_gb300 import VBCSR, lib
    w = syn.tiny_multispecies(0)
    H = VBCSR.from_pattern(w.pattern, w.values, torch.float64, "cuda:0")
    H.set_schedule("bucketed", 2, mma_staged=True, scalar_kernel=False, value_ring=False)
    t = H.get_tuning()
    assert (t["schedule"], t["mma_staged"], t["scalar_kernel"], t["value_ring"]) == ("bucketed", True, False, False)
    H.set_schedule("persistent")
    H.apply_tuning(t)
    assert H.get_tuning()["value_ring"] is False and H.get_tuning()["scalar_kernel"] is False
    for bad in (32, -1):
        assert lib().vbcsr_set_schedule(H.handle, bad, 0) != 0
    assert lib().vbcsr_set_schedule(H.handle, 1, 3) != 0
    assert lib().vbcsr_set_schedule(H.handle, 1 | 2 | 4 | 8 | 16, 4) == 0
    H.set_schedule("persistent", pipelined_f32=False)
    assert H.get_tuning()["pipelined_f32"] is False


def test_full_size_batched_workload_every_element():
    """The batched workload at full size: 256 structures of 50-2000 atoms
    (log-uniform, b in {4, 9, 13}, 5 A cutoff), FP32, k = 8, in its autotuned
    schedule and replayed from a captured CUDA graph: every output element
    against the per-structure oracle (FP64 on the FP32-rounded inputs)."""
    import os
    w, H, vals = _batched(n_structs=256, n_max=2000, seed=0)
    assert H.info.n_structs == 256
    k = 8
    X = np.random.default_rng(0).standard_normal((w.pattern.n_cols, k)).astype(np.float32).astype(np.float64)
    Xd = torch.from_numpy(X).float().cuda()
    nth = os.cpu_count() or 1
    voff = w.pattern.value_offset()
    coff = np.concatenate([[0], np.cumsum(w.pattern.col_bsize.astype(np.int64))])
    sref, sabs = [], []
    for s, part in enumerate(w.parts):
        b0, b1 = w.struct_brow_offsets[s], w.struct_brow_offsets[s + 1]
        v = vals[voff[w.pattern.block_row_ptr[b0]]:voff[w.pattern.block_row_ptr[b1]]]
        Xs = X[coff[b0]:coff[b1]]
        sref.append(oracle.spmm(part, v, Xs, nthreads=nth))
        sabs.append(oracle.spmm(part, np.abs(v), np.abs(Xs), nthreads=nth))
    ref, scale = np.concatenate(sref), np.concatenate(sabs)
    H.autotune(k)
    got = H.spmm(Xd).cpu().numpy().astype(np.float64)
    assert rel_fro(got, ref) <= TOL_MIXED
    check_elementwise(got, ref, scale, 1e-4)
    Y = torch.empty(w.pattern.n_rows, k, dtype=torch.float32, device="cuda:0")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        H.spmm(Xd, 1.0, 0.0, Y)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        H.spmm(Xd, 1.0, 0.0, Y)
    Y.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(Y.cpu().numpy().astype(np.float64), got)

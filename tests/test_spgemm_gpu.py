"""GPU parity of the thresholded block sparse product (Eqs. 2-3) against the
oracle: the kept pattern exactly, the values within the FP64 tolerance."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as syn
from synthetic.structures import BlockPattern
from _parity import TOL_F64, rel_fro

pytestmark = pytest.mark.gpu


def _h(pat, vals, dtype=torch.float64):
    from paper_2609_04397_gb300 import VBCSR
    return VBCSR.from_pattern(pat, vals, dtype, "cuda:0")


def _check(C, ref, tol=TOL_F64):
    rb, cb, ptr, cols, vals = ref
    crb, ccb, cptr, ccol = C.pattern
    assert np.array_equal(crb, rb) and np.array_equal(ccb, cb)
    assert np.array_equal(cptr, ptr) and np.array_equal(ccol, cols)
    got = C.get_values().cpu().numpy().astype(np.float64)
    assert rel_fro(got, vals) <= tol
    scale = np.abs(vals).max() if len(vals) else 1.0
    assert np.abs(got - vals).max() <= 10 * tol * scale


@pytest.mark.parametrize("eps", [0.0, 0.3, 2.0])
def test_spgemm_rectangular_random(eps):
    pa = syn.random_pattern(23, 17, (1, 3, 4, 9), 0.25, 61, empty_rows=2, unsorted=True)
    pb = syn.random_pattern(17, 19, (2, 5, 13), 0.25, 62, empty_rows=2, unsorted=True)
    pb = BlockPattern(pa.col_bsize, pb.col_bsize, pb.block_row_ptr, pb.block_col_idx)
    va, vb = syn.random_values(pa, 61), syn.random_values(pb, 62)
    C = _h(pa, va).spgemm(_h(pb, vb), eps)
    _check(C, oracle.spgemm(pa, va, pb, vb, eps))


def test_spgemm_square_of_multispecies_operator():
    w = syn.tiny_multispecies(0)
    H = _h(w.pattern, w.values)
    for eps in (0.0, 0.05):
        _check(H.spgemm(H, eps), oracle.spgemm(w.pattern, w.values, w.pattern, w.values, eps))


def test_spgemm_result_is_an_operator():
    """The product handle multiplies like (A B) X."""
    pa = syn.random_pattern(20, 20, (4, 9), 0.2, 63)
    pa = BlockPattern(pa.row_bsize, pa.row_bsize, pa.block_row_ptr, pa.block_col_idx)
    va = syn.random_values(pa, 63)
    H = _h(pa, va)
    C = H.spgemm(H)
    X = torch.randn(pa.n_cols, 5, dtype=torch.float64, device="cuda:0")
    assert torch.allclose(C.spmm(X), H.spmm(H.spmm(X)), rtol=1e-12, atol=1e-12)


def test_spgemm_fp32():
    pa = syn.random_pattern(18, 18, (4, 9, 13), 0.25, 64)
    pa = BlockPattern(pa.row_bsize, pa.row_bsize, pa.block_row_ptr, pa.block_col_idx)
    va = syn.random_values(pa, 64).astype(np.float32)
    C = _h(pa, va, torch.float32).spgemm(_h(pa, va, torch.float32), 0.5)
    ref = oracle.spgemm(pa, va.astype(np.float64), pa, va.astype(np.float64), 0.5)
    rb, cb, ptr, cols, vals = ref
    got = C.get_values().cpu().numpy().astype(np.float64)
    # FP32 arithmetic: compare on the blocks both kept (a block right at eps may differ)
    crb, ccb, cptr, ccol = C.pattern
    assert abs(len(ccol) - len(cols)) <= 2
    if np.array_equal(ccol, cols):
        assert rel_fro(got, vals) <= 1e-5


def test_spgemm_rejects_mismatched_inner_sizes():
    from paper_2609_04397_gb300 import VBCSRError
    pa = syn.random_pattern(5, 4, (2,), 0.5, 1)
    pb = syn.random_pattern(4, 3, (3,), 0.5, 2)
    with pytest.raises(VBCSRError):
        _h(pa, syn.random_values(pa, 1)).spgemm(_h(pb, syn.random_values(pb, 2)))

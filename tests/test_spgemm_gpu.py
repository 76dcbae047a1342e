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


def test_spgemm_row_beyond_the_shared_table():
    """A block row with more candidate blocks than the symbolic stage's
    shared-memory table holds goes through its device-memory workspace and
    gives the same result."""
    rng = np.random.default_rng(65)
    na, nk, nj = 6, 700, 1500
    # row 0 of A is dense; B is sparse with ~3 blocks per row: row 0 of C has ~1300 candidates
    a_ptr = [0, nk] + [nk + 3 * r for r in range(1, na)]
    a_col = list(range(nk)) + [int(c) for r in range(1, na) for c in sorted(rng.choice(nk, 3, replace=False))]
    b_ptr = [3 * r for r in range(nk + 1)]
    b_col = [int(c) for r in range(nk) for c in sorted(rng.choice(nj, 3, replace=False))]
    pa = BlockPattern(np.array([2, 1, 3, 2, 1, 2], np.int32), np.ones(nk, np.int32),
                      np.array(a_ptr, np.int64), np.array(a_col, np.int32))
    pb = BlockPattern(np.ones(nk, np.int32), rng.integers(1, 3, nj).astype(np.int32),
                      np.array(b_ptr, np.int64), np.array(b_col, np.int32))
    va, vb = syn.random_values(pa, 65), syn.random_values(pb, 66)
    for eps in (0.0, 0.5):
        C = _h(pa, va).spgemm(_h(pb, vb), eps)
        _check(C, oracle.spgemm(pa, va, pb, vb, eps))


def test_spgemm_zincblende_and_repeatable():
    """Square of a small zinc-blende operator at a threshold that drops about
    half of the blocks; a second call gives the identical pattern and values."""
    w = syn.zincblende(150)
    H = _h(w.pattern, w.values)
    ref = oracle.spgemm(w.pattern, w.values, w.pattern, w.values, 0.0)
    _check(H.spgemm(H, 0.0), ref)
    rb, cb, ptr, cols, vals = ref
    rows = np.repeat(np.arange(len(rb)), np.diff(ptr))
    sz = rb[rows].astype(np.int64) * cb[cols]
    norms = np.sqrt(np.add.reduceat(vals * vals, np.concatenate([[0], np.cumsum(sz)[:-1]])))
    eps = float(np.median(norms))
    C1, C2 = H.spgemm(H, eps), H.spgemm(H, eps)
    _check(C1, oracle.spgemm(w.pattern, w.values, w.pattern, w.values, eps))
    assert all(np.array_equal(x, y) for x, y in zip(C1.pattern, C2.pattern))
    assert torch.equal(C1.get_values(), C2.get_values())


def test_spgemm_everything_dropped_and_empty_operands():
    """A threshold above every bound keeps nothing; an operand without blocks
    gives an empty product. Both results are valid operators."""
    w = syn.tiny_multispecies(0)
    H = _h(w.pattern, w.values)
    C = H.spgemm(H, 1e30)
    assert C.info.nblk == 0 and C.nnz == 0
    X = torch.randn(C.shape[1], 3, dtype=torch.float64, device="cuda:0")
    assert torch.count_nonzero(C.spmm(X)) == 0
    pe = BlockPattern(w.pattern.row_bsize, w.pattern.col_bsize,
                      np.zeros(len(w.pattern.row_bsize) + 1, np.int64), np.zeros(0, np.int32))
    E = _h(pe, np.zeros(0))
    for P in (E.spgemm(H), H.spgemm(E)):
        assert P.info.nblk == 0

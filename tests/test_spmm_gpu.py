"""GPU parity of the FP64 / FP32 forward product, adjoint and pattern-sampled
product against the CPU oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as syn
from synthetic.structures import BlockPattern
from _parity import (TOL_F64, TOL_MIXED, adjoint_ref, check_elementwise, forward_ref, rel_fro,
                     sddmm_ref)

pytestmark = pytest.mark.gpu


def _handle(pat, vals, dtype=torch.float64):
    from paper_2609_04397_gb300 import VBCSR
    return VBCSR.from_pattern(pat, vals, dtype, "cuda:0")


def _dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dtype)


def _run_forward(H, pat, vals, k, alpha, beta, ld_extra=0, seed=0, precision="native", tol=TOL_F64):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((pat.n_cols, k + ld_extra))
    Y0 = rng.standard_normal((pat.n_rows, k + ld_extra))
    Xd = _dev(X, H.dtype)[:, :k]
    Yd = _dev(Y0, H.dtype)
    H.spmm(Xd, alpha, beta, Yd[:, :k], precision=precision)
    got = Yd.cpu().numpy()
    Xc = X[:, :k].astype(np.float32).astype(np.float64) if H.dtype == torch.float32 else X[:, :k]
    Y0c = Y0[:, :k].astype(np.float32).astype(np.float64) if H.dtype == torch.float32 else Y0[:, :k]
    ref, scale = forward_ref(pat, vals, Xc, alpha, beta, Y0c)
    assert rel_fro(got[:, :k], ref) <= tol
    check_elementwise(got[:, :k], ref, scale, tol)
    # columns beyond k (inside the leading dimension) are untouched
    if ld_extra:
        assert np.array_equal(got[:, k:], Y0[:, k:].astype(got.dtype))


def test_tiny_multispecies_forward():
    """200 atoms, b in {4, 9}, X 1300 x 8 N(0,1), seed 0."""
    w = syn.tiny_multispecies(0)
    H = _handle(w.pattern, w.values)
    X = syn.normal_panel(w.pattern.n_cols, 8, 0)
    Y = H.spmm(_dev(X)).cpu().numpy()
    ref, scale = forward_ref(w.pattern, w.values, X, 1.0, 0.0, None)
    assert rel_fro(Y, ref) <= TOL_F64
    check_elementwise(Y, ref, scale, TOL_F64)
    for alpha, beta in ((2.0, -1.0), (-1.0, 1.0), (0.0, 1.0), (1.0, 0.0)):
        _run_forward(H, w.pattern, w.values, 8, alpha, beta)
    H.check()


SIZES = [(1, 2, 3), (4, 9, 13), (1, 5, 16), (17, 3, 20), (7, 8, 9, 10, 11, 12)]


@pytest.mark.parametrize("schedule", ["persistent", "bucketed"])
@pytest.mark.parametrize("sizes", SIZES)
@pytest.mark.parametrize("k", [1, 2, 3, 7, 8, 16, 32, 33])
def test_random_patterns_forward_adjoint(sizes, k, schedule):
    """Both launch schedules: one persistent launch over every item (the
    default) and one launch per row count."""
    seed = hash((sizes, k)) % 1000
    pat = syn.random_pattern(37, 29, sizes, 0.15, seed, empty_rows=3, unsorted=True)
    vals = syn.random_values(pat, seed)
    H = _handle(pat, vals)
    H.set_schedule(schedule)
    for alpha, beta in ((1.0, 0.0), (-1.0, 1.0), (2.0, -1.0), (0.0, -1.0), (0.5, 0.25)):
        _run_forward(H, pat, vals, k, alpha, beta, ld_extra=(k % 3), seed=seed)
        rng = np.random.default_rng(seed + 1)
        X = rng.standard_normal((pat.n_rows, k))
        Y0 = rng.standard_normal((pat.n_cols, k))
        Yd = _dev(Y0)
        H.spmm_adjoint(_dev(X), alpha, beta, Yd)
        ref, scale = adjoint_ref(pat, vals, X, alpha, beta, Y0)
        got = Yd.cpu().numpy()
        assert rel_fro(got, ref) <= TOL_F64
        check_elementwise(got, ref, scale, TOL_F64)
    H.check()


@pytest.mark.parametrize("k", [1, 5, 8, 40])
def test_sddmm_random(k):
    pat = syn.random_pattern(31, 23, (1, 4, 9, 13, 17), 0.2, 5 + k, empty_rows=2, unsorted=True)
    H = _handle(pat, syn.random_values(pat, 5))
    rng = np.random.default_rng(k)
    A = rng.standard_normal((pat.n_rows, k))
    B = rng.standard_normal((pat.n_cols, k))
    D0 = rng.standard_normal(pat.nnz)
    for alpha, beta in ((1.0, 0.0), (2.0, -1.0), (0.0, 0.5)):
        Dd = _dev(D0)
        H.sddmm(_dev(A), _dev(B), alpha, beta, Dd)
        ref, scale = sddmm_ref(pat, A, B, alpha, beta, D0)
        got = Dd.cpu().numpy()
        assert rel_fro(got, ref) <= TOL_F64
        check_elementwise(got, ref, scale, TOL_F64)


def test_wide_rows_and_tall_blocks():
    """Block sizes above 16 (row chunking) and panels wider than the staged
    shared-memory window (K > 512) in both directions."""
    pat = syn.random_pattern(9, 11, (33, 60, 150), 0.6, 3)
    vals = syn.random_values(pat, 3)
    H = _handle(pat, vals)
    for k in (1, 8, 33):
        _run_forward(H, pat, vals, k, 1.0, 0.5, seed=k)
        X = np.random.default_rng(k).standard_normal((pat.n_rows, k))
        got = H.spmm_adjoint(_dev(X)).cpu().numpy()
        ref, scale = adjoint_ref(pat, vals, X, 1.0, 0.0, None)
        check_elementwise(got, ref, scale, TOL_F64)
    # the pattern-sampled product over the same rows (chunked rows, wide windows,
    # several staged column chunks of A and B, leading dimensions above k)
    for k in (1, 70):
        rng = np.random.default_rng(k + 100)
        A = rng.standard_normal((pat.n_rows, k + 3))
        B = rng.standard_normal((pat.n_cols, k + 5))
        D0 = rng.standard_normal(pat.nnz)
        Dd = _dev(D0)
        H.sddmm(_dev(A)[:, :k], _dev(B)[:, :k], 1.5, -0.5, Dd)
        ref, scale = sddmm_ref(pat, A[:, :k], B[:, :k], 1.5, -0.5, D0)
        check_elementwise(Dd.cpu().numpy(), ref, scale, TOL_F64)


def test_sddmm_fp32_operator():
    pat = syn.random_pattern(30, 30, (4, 9, 13), 0.2, 11)
    H = _handle(pat, syn.random_values(pat, 11).astype(np.float32), torch.float32)
    rng = np.random.default_rng(11)
    for k in (1, 16, 40):
        A = rng.standard_normal((pat.n_rows, k)).astype(np.float32)
        B = rng.standard_normal((pat.n_cols, k)).astype(np.float32)
        got = H.sddmm(_dev(A, torch.float32), _dev(B, torch.float32)).cpu().numpy().astype(np.float64)
        ref, scale = sddmm_ref(pat, A.astype(np.float64), B.astype(np.float64), 1.0, 0.0, None)
        check_elementwise(got, ref, scale, 1e-5)


def test_beta_zero_and_alpha_zero_do_not_read():
    pat = syn.random_pattern(20, 20, (3, 9), 0.3, 4)
    vals = syn.random_values(pat, 4)
    H = _handle(pat, vals)
    X = _dev(np.random.default_rng(0).standard_normal((pat.n_cols, 4)))
    Y = torch.full((pat.n_rows, 4), float("nan"), dtype=torch.float64, device="cuda:0")
    H.spmm(X, 1.0, 0.0, Y)
    assert torch.isfinite(Y).all()
    Xn = torch.full_like(X, float("nan"))
    Y2 = torch.ones((pat.n_rows, 4), dtype=torch.float64, device="cuda:0")
    H.spmm(Xn, 0.0, 3.0, Y2)
    assert torch.equal(Y2, torch.full_like(Y2, 3.0))


def test_degenerate_sizes():
    from paper_2609_04397_gb300 import VBCSR
    # no blocks at all
    pat = BlockPattern(np.array([2, 3]), np.array([4]), np.array([0, 0, 0]), np.zeros(0))
    H = VBCSR.from_pattern(pat, np.zeros(0), torch.float64, "cuda:0")
    Y = torch.full((5, 3), 7.0, dtype=torch.float64, device="cuda:0")
    H.spmm(torch.ones((4, 3), dtype=torch.float64, device="cuda:0"), 1.0, 0.5, Y)
    assert torch.equal(Y, torch.full_like(Y, 3.5))
    # k = 0 launches nothing
    H.spmm(torch.ones((4, 0), dtype=torch.float64, device="cuda:0"), 1.0, 0.0,
           torch.ones((5, 0), dtype=torch.float64, device="cuda:0"))
    # zero block rows
    pat0 = BlockPattern(np.zeros(0), np.array([2]), np.array([0]), np.zeros(0))
    H0 = VBCSR.from_pattern(pat0, np.zeros(0), torch.float64, "cuda:0")
    assert H0.shape == (0, 2)
    H.check()


def test_alias_rejected():
    from paper_2609_04397_gb300 import VBCSRError
    w = syn.tiny_multispecies(0)
    H = _handle(w.pattern, w.values)
    X = torch.ones((1300, 4), dtype=torch.float64, device="cuda:0")
    with pytest.raises(VBCSRError) as ei:
        H.spmm(X, 1.0, 0.0, X)
    assert ei.value.status == -7


def test_values_roundtrip_and_update():
    pat = syn.random_pattern(25, 25, (4, 9, 13), 0.2, 6, unsorted=True)
    vals = syn.random_values(pat, 6)
    H = _handle(pat, vals)
    assert np.array_equal(H.get_values().cpu().numpy(), vals)
    v2 = syn.random_values(pat, 7)
    H.set_values(_dev(v2))
    assert np.array_equal(H.get_values().cpu().numpy(), v2)
    H.set_values(v2 * 2.0)       # host path
    assert np.array_equal(H.get_values().cpu().numpy(), v2 * 2.0)
    _run_forward(H, pat, v2 * 2.0, 5, 1.0, 0.0)


def test_shape_class_registry():
    w = syn.tiny_multispecies(0)
    H = _handle(w.pattern, w.values)
    cls = H.shape_classes()
    pat = w.pattern
    rows = pat.block_rows()
    expect = {}
    for bi, bj in zip(pat.row_bsize[rows], pat.col_bsize[pat.block_col_idx]):
        expect[(int(bi), int(bj))] = expect.get((int(bi), int(bj)), 0) + 1
    assert {(a, b): c for a, b, c in cls} == expect
    assert len(cls) == 4
    assert [(a, b) for a, b, _ in cls] == sorted(expect)          # increasing (b_i, b_j)
    # rectangular, unsorted rows, many sizes on both sides
    pat = syn.random_pattern(60, 45, (1, 2, 5, 7, 13, 16, 20), 0.2, 9, empty_rows=3, unsorted=True)
    H = _handle(pat, syn.random_values(pat, 9))
    cls = H.shape_classes()
    expect = {}
    for bi, bj in zip(pat.row_bsize[pat.block_rows()], pat.col_bsize[pat.block_col_idx]):
        expect[(int(bi), int(bj))] = expect.get((int(bi), int(bj)), 0) + 1
    assert [(a, b, c) for a, b, c in cls] == [(a, b, expect[(a, b)]) for a, b in sorted(expect)]


def test_fp32_operator():
    pat = syn.random_pattern(40, 40, (4, 9, 13), 0.15, 8)
    vals = syn.random_values(pat, 8)
    v32 = vals.astype(np.float32)
    H = _handle(pat, v32, torch.float32)
    _run_forward(H, pat, v32.astype(np.float64), 8, 1.0, 0.0, tol=TOL_MIXED)
    _run_forward(H, pat, v32.astype(np.float64), 3, 2.0, -1.0, tol=TOL_MIXED)


def test_f32_mode_on_fp64_operator():
    w = syn.tiny_multispecies(0)
    H = _handle(w.pattern, w.values)
    _run_forward(H, w.pattern, w.values, 8, 1.0, 0.0, precision="f32", tol=TOL_MIXED)


@pytest.mark.parametrize("kc,warps", [(1, 1), (4, 2), (8, 8), (32, 4), (16, 1)])
def test_tuning_variants_agree(kc, warps):
    w = syn.tiny_multispecies(0)
    H = _handle(w.pattern, w.values)
    H.set_tuning(kc, warps)
    _run_forward(H, w.pattern, w.values, 11, 1.0, 0.0)


def test_zincblende_full_size_sampled_rows():
    """~50k-atom zinc-blende cluster (549,607 rows, 1.67e8 entries) at k = 1, 8
    and 32: every output of 64 sampled block rows against the oracle."""
    w = syn.zincblende(50_000)
    pat = w.pattern
    H = _handle(pat, w.values)
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(pat.n_brows, 64, replace=False))
    roff = np.concatenate([[0], np.cumsum(pat.row_bsize.astype(np.int64))])
    for k in (1, 8, 32):
        X = syn.normal_panel(pat.n_cols, k, 0)
        Y = H.spmm(_dev(X)).cpu().numpy()
        ref = np.zeros_like(Y)
        scale = np.zeros_like(Y)
        absv, absx = np.abs(w.values), np.abs(X)
        for i in rows:
            ref = oracle.spmm(pat, w.values, X, row_range=(i, i + 1), Y=ref, beta=1.0)
            scale = oracle.spmm(pat, absv, absx, row_range=(i, i + 1), Y=scale, beta=1.0)
        sel = np.concatenate([np.arange(roff[i], roff[i + 1]) for i in rows])
        check_elementwise(Y[sel], ref[sel], scale[sel], TOL_F64)
        assert rel_fro(Y[sel], ref[sel]) <= TOL_F64
    H.check()


@pytest.mark.parametrize("sizes,precision", [((4, 9, 13), "native"), ((1,), "native"), ((1,), "df32"),
                                              ((1,), "f32")])
@pytest.mark.parametrize("transpose", [False, True])
def test_fused_epilogue_gamma_z_and_dot(transpose, sizes, precision):
    """Y = alpha op(H) X + beta Y + gamma Z and dot = sum(R * Y) through
    vbcsr_spmm_ex, on a variable-block operator and on a scalar one (whose
    forward product runs in the scalar kernel, in each arithmetic kind)."""
    n = 33 if sizes != (1,) else 200
    pat = syn.random_pattern(n, n, sizes, 0.2, 21)
    vals = syn.random_values(pat, 21)
    H = _handle(pat, vals)
    rng = np.random.default_rng(3)
    n_in, n_out = (pat.n_rows, pat.n_cols) if transpose else (pat.n_cols, pat.n_rows)
    X = rng.standard_normal((n_in, 5))
    Y0 = rng.standard_normal((n_out, 5))
    Z = rng.standard_normal((n_out, 5))
    R = rng.standard_normal((n_out, 5))
    Yd = _dev(Y0)
    dot = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    H.spmm_ex(_dev(X), 2.0, -1.0, Yd, transpose=transpose, gamma=0.5, Z=_dev(Z), R=_dev(R), dot_out=dot,
              precision=precision)
    fn = oracle.spmm_adjoint if transpose else oracle.spmm
    ref = fn(pat, vals, X, 2.0, -1.0, Y0) + 0.5 * Z
    got = Yd.cpu().numpy()
    tol = TOL_MIXED if precision == "f32" else TOL_F64
    assert rel_fro(got, ref) <= tol
    # the dot is of the stored Y: exact to FP64 rounding of the sum in every mode
    assert abs(dot.item() - np.sum(R * got)) <= 1e-12 * np.sum(np.abs(R * got))


@pytest.mark.parametrize("sizes", SIZES + [(3, 16), (8,)])
@pytest.mark.parametrize("k", [1, 8, 33])
def test_df32_mode_meets_fp64_tolerance(sizes, k):
    """FP64 operands in double-FP32 arithmetic: held to the FP64 tolerance.
    Operators with one or two row counts run the persistent kernel's wide
    form (four columns per lane up to 13 rows), the others its narrow form."""
    seed = 7 + k
    pat = syn.random_pattern(37, 29, sizes, 0.15, seed, empty_rows=3, unsorted=True)
    vals = syn.random_values(pat, seed)
    H = _handle(pat, vals)
    for alpha, beta in ((1.0, 0.0), (2.0, -1.0)):
        _run_forward(H, pat, vals, k, alpha, beta, ld_extra=1, seed=seed, precision="df32")
        X = np.random.default_rng(seed).standard_normal((pat.n_rows, k))
        got = H.spmm_adjoint(_dev(X), precision="df32").cpu().numpy()
        ref, scale = adjoint_ref(pat, vals, X, 1.0, 0.0, None)
        assert rel_fro(got, ref) <= TOL_F64
        check_elementwise(got, ref, scale, TOL_F64)


def test_df32_mode_zincblende_sampled_rows():
    w = syn.zincblende(8000)
    pat = w.pattern
    H = _handle(pat, w.values)
    X = syn.normal_panel(pat.n_cols, 16, 0)
    got = H.spmm(_dev(X), precision="df32").cpu().numpy()
    ref, scale = forward_ref(pat, w.values, X, 1.0, 0.0, None)
    assert rel_fro(got, ref) <= TOL_F64
    check_elementwise(got, ref, scale, TOL_F64)
    # and the FP32 copy is not what it used: the plain FP32 mode is far less accurate
    got32 = H.spmm(_dev(X), precision="f32").cpu().numpy()
    assert rel_fro(got32, ref) > 100 * rel_fro(got, ref)


def test_backend_selection():
    w = syn.tiny_multispecies(0)
    assert _handle(w.pattern, w.values).backend == "vbcsr"
    n = 50
    rng = np.random.default_rng(0)
    mask = rng.random((n, n)) < 0.1
    np.fill_diagonal(mask, True)
    ptr = np.concatenate([[0], np.cumsum(mask.sum(1))])
    cols = np.concatenate([np.nonzero(mask[i])[0] for i in range(n)])
    for b, name in ((1, "csr"), (8, "bsr")):
        pat = BlockPattern(np.full(n, b), np.full(n, b), ptr, cols)
        assert _handle(pat, syn.random_values(pat, 1)).backend == name


@pytest.mark.parametrize("density", [0.02, 0.2, 0.6, 1.0])
@pytest.mark.parametrize("k", [1, 3, 8, 9, 17])
def test_csr_backend_scalar_kernel(density, k):
    """Scalar operators (all blocks 1 x 1) through the scalar kernel, against
    the oracle and against the block-row kernels on the same operator. The
    densities give ~12, ~120, ~360 and 600 entries per row, so every lane
    count the kernel picks from the row length (2, 4, 8 for FP64 and
    double-FP32; 4, 8, 16, 32 for the FP32 kinds) runs."""
    pat = syn.random_pattern(300, 600, (1,), density, 90 + k, empty_rows=7, unsorted=True)
    vals = syn.random_values(pat, 90 + k)
    H = _handle(pat, vals)
    assert H.backend == "csr"
    for alpha, beta in ((1.0, 0.0), (2.0, -1.0), (0.0, 0.5)):
        _run_forward(H, pat, vals, k, alpha, beta, ld_extra=1, seed=k)
    Xh = np.random.default_rng(k).standard_normal((pat.n_cols, k))
    X = _dev(Xh)
    Ys = H.spmm(X)
    H.set_schedule("bucketed", scalar_kernel=False)
    Yb = H.spmm(X)
    # the two kernels sum a row in different orders: they agree to the
    # forward-error scale of a reordered dot product, 1e-12 (|H| |X|)
    _, scale = forward_ref(pat, vals, Xh, 1.0, 0.0, None)
    check_elementwise(Ys.cpu().numpy(), Yb.cpu().numpy(), scale, TOL_F64)
    H32 = _handle(pat, vals.astype(np.float32), torch.float32)
    _run_forward(H32, pat, vals.astype(np.float32).astype(np.float64), k, 1.0, 0.0, tol=TOL_MIXED)
    # the FP64-accurate double-FP32 mode and FP32 products run in the scalar kernel too
    H.set_schedule("bucketed")
    _run_forward(H, pat, vals, k, 2.0, -1.0, ld_extra=1, seed=k + 1, precision="df32")
    Y0 = np.random.default_rng(k + 2).standard_normal((pat.n_rows, k))
    Yd = _dev(Y0)
    H.spmm(X, 2.0, -1.0, Yd, precision="f32")
    ref, scale = forward_ref(pat, vals, Xh, 2.0, -1.0, Y0)
    assert rel_fro(Yd.cpu().numpy(), ref) <= TOL_MIXED
    check_elementwise(Yd.cpu().numpy(), ref, scale, 1e-4)
    # and the tensor-core modes, whose piece products run in the scalar kernel
    for mode in ("tf32x3", "bf16x2"):
        Yd = _dev(Y0)
        H.spmm(X, 2.0, -1.0, Yd, precision=mode)
        assert rel_fro(Yd.cpu().numpy(), ref) <= TOL_MIXED
        check_elementwise(Yd.cpu().numpy(), ref, scale, 1e-4)


@pytest.mark.parametrize("precision", ["native", "f32", "df32", "bf16x2", "tf32x3"])
def test_many_column_passes(precision):
    """k = 100: several passes of 32 output columns (the last one 4 wide) in
    every kernel form (the value rings, the tensor-core tiles), forward and
    adjoint, with leading dimensions above k."""
    pat = syn.random_pattern(30, 26, (3, 9, 13, 17), 0.25, 91, empty_rows=2, unsorted=True)
    vals = syn.random_values(pat, 91)
    H = _handle(pat, vals)
    rng = np.random.default_rng(91)
    k = 100
    X = rng.standard_normal((pat.n_cols, k + 3))
    got = H.spmm(_dev(X)[:, :k], precision=precision).cpu().numpy()
    ref, scale = forward_ref(pat, vals, X[:, :k], 1.0, 0.0, None)
    tol = TOL_F64 if precision in ("native", "df32") else 1e-4
    check_elementwise(got, ref, scale, tol)
    Xa = rng.standard_normal((pat.n_rows, k))
    got = H.spmm_adjoint(_dev(Xa), precision=precision).cpu().numpy()
    ref, scale = adjoint_ref(pat, vals, Xa, 1.0, 0.0, None)
    check_elementwise(got, ref, scale, tol)


def test_one_launch_per_product_under_the_persistent_schedule():
    """The bench counts one kernel launch per FP64 product (the default
    persistent schedule); a profiler trace of one product shows exactly one
    kernel of the library."""
    from torch.profiler import ProfilerActivity, profile
    w = syn.tiny_multispecies(0)
    H = _handle(w.pattern, w.values)
    X = _dev(syn.normal_panel(w.pattern.n_cols, 8, 0))
    Y = torch.empty(w.pattern.n_rows, 8, dtype=torch.float64, device="cuda:0")
    H.spmm(X, 1.0, 0.0, Y)
    torch.cuda.synchronize()
    kernels = []
    for _ in range(2):   # the first trace of a process can come back before its activity buffers fill
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            H.spmm(X, 1.0, 0.0, Y)
            torch.cuda.synchronize()
        kernels = [e.name for e in prof.events() if e.device_type == torch.autograd.DeviceType.CUDA
                   and "vbcsr" in e.name]
        if kernels:
            break
    assert len(kernels) == 1 and "fma_persistent_kernel" in kernels[0], kernels


def test_registry_with_very_many_block_sizes():
    """More than 2^20 (row size, column size) combinations take the planner's
    ordered-map registry instead of its dense count table: 1100 distinct row
    sizes, 1000 distinct column sizes, a few blocks among them."""
    nr, nc = 1100, 1000
    rb = np.arange(1, nr + 1, dtype=np.int32)
    cb = np.arange(1, nc + 1, dtype=np.int32)
    rng = np.random.default_rng(5)
    rows = np.sort(rng.choice(40, 12, replace=False))          # small rows and columns keep the values small
    ptr = np.zeros(nr + 1, np.int64)
    cols = []
    for i in range(nr):
        if i in rows:
            cols.extend(sorted(rng.choice(30, 2, replace=False).tolist()))
        ptr[i + 1] = len(cols)
    pat = BlockPattern(rb, cb, ptr, np.array(cols, np.int32))
    vals = syn.random_values(pat, 5)
    H = _handle(pat, vals)
    expect = {}
    for bi, bj in zip(pat.row_bsize[pat.block_rows()], pat.col_bsize[pat.block_col_idx]):
        expect[(int(bi), int(bj))] = expect.get((int(bi), int(bj)), 0) + 1
    assert H.shape_classes() == [(a, b, expect[(a, b)]) for a, b in sorted(expect)]
    X = np.random.default_rng(6).standard_normal((pat.n_cols, 2))
    got = H.spmm(_dev(X)).cpu().numpy()
    ref, scale = forward_ref(pat, vals, X, 1.0, 0.0, None)
    check_elementwise(got, ref, scale, TOL_F64)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("schedule", ["persistent", "bucketed"])
@pytest.mark.parametrize("b", [4, 8, 13])
def test_bsr_backend_native(b, schedule, dtype):
    """Uniform-block operators (the BSR backend) in the operator's own
    arithmetic, FP64 and FP32, forward and adjoint, element by element against
    the oracle at k = 1, 3, 8, 16, 33 (FP32 operators at the FP32 tolerance)."""
    pat = syn.random_pattern(70, 70, (b,), 0.12, 40 + b, empty_rows=2, unsorted=True)
    vals = syn.random_values(pat, 40 + b)
    if dtype == torch.float32:
        vals = vals.astype(np.float32).astype(np.float64)
    H = _handle(pat, vals, dtype)
    assert H.backend == "bsr"
    H.set_schedule(schedule)
    tol = TOL_F64 if dtype == torch.float64 else TOL_MIXED
    for k in (1, 3, 8, 16, 33):
        _run_forward(H, pat, vals, k, 1.0, 0.0, seed=k, tol=tol)
        _run_forward(H, pat, vals, k, -0.5, 2.0, ld_extra=3, seed=k + 1, tol=tol)
        Xa = np.random.default_rng(k).standard_normal((pat.n_rows, k))
        if dtype == torch.float32:
            Xa = Xa.astype(np.float32).astype(np.float64)
        got = H.spmm_adjoint(_dev(Xa, dtype)).cpu().numpy()
        ref, scale = adjoint_ref(pat, vals, Xa, 1.0, 0.0, None)
        check_elementwise(got, ref, scale, tol)


@pytest.mark.parametrize("kind", ["bsr", "vbcsr"])
def test_structural_domain_full_size_sampled_rows(kind):
    """The ~500 MiB structural domains of the kernel benchmark (Sec. IV; BSR
    b = 8 and variable blocks b in [9, 20]) at k = 1 and 16, FP64 and
    double-FP32 products: every output of 64 sampled block rows against the
    oracle."""
    w = syn.domain(kind)
    pat = w.pattern
    H = _handle(pat, w.values)
    assert H.backend == kind
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(pat.n_brows, 64, replace=False))
    roff = np.concatenate([[0], np.cumsum(pat.row_bsize.astype(np.int64))])
    sel = np.concatenate([np.arange(roff[i], roff[i + 1]) for i in rows])
    absv = np.abs(w.values)
    for k in (1, 16):
        X = syn.normal_panel(pat.n_cols, k, 0)
        ref = np.zeros((pat.n_rows, k))
        scale = np.zeros((pat.n_rows, k))
        for i in rows:
            ref = oracle.spmm(pat, w.values, X, row_range=(i, i + 1), Y=ref, beta=1.0)
            scale = oracle.spmm(pat, absv, np.abs(X), row_range=(i, i + 1), Y=scale, beta=1.0)
        for precision in ("native", "df32"):
            Y = H.spmm(_dev(X), precision=precision).cpu().numpy()
            check_elementwise(Y[sel], ref[sel], scale[sel], TOL_F64)
            assert rel_fro(Y[sel], ref[sel]) <= TOL_F64
    H.check()


@pytest.mark.parametrize("k,ld", [(8, 8), (12, 12), (12, 16), (16, 16), (20, 24), (32, 32), (33, 36), (40, 40),
                                  (16, 18)])
@pytest.mark.parametrize("prec,dtype", [("native", torch.float32), ("f32", torch.float64)])
def test_pipelined_fp32_kernel(k, ld, prec, dtype):
    """FP32 values at k >= 8 under the persistent schedule (the pipelined
    CUDA-core kernel: 4-row register tiles fed from a shared-memory ring),
    element by element against the oracle on FP32-rounded inputs: rows of
    every height (1 to 20, rows above 16 cut into items), panels wider than one
    512-column window, several column passes (k > 32), leading dimensions
    above k (a multiple of 4; ld = 18 takes the other kernel), alpha / beta,
    and the fused gamma Z and dot epilogue."""
    pat = syn.random_pattern(50, 47, (1, 4, 9, 13, 16, 20), 0.2, 60 + k, empty_rows=2, unsorted=True)
    wide = syn.random_pattern(3, 60, (13,), 0.9, 61, empty_rows=0)
    vals = syn.random_values(pat, 60 + k).astype(np.float32).astype(np.float64)
    for p, v in ((pat, vals), (wide, syn.random_values(wide, 62).astype(np.float32).astype(np.float64))):
        H = _handle(p, v, dtype)
        H.set_schedule("persistent")
        rng = np.random.default_rng(k)
        X = rng.standard_normal((p.n_cols, ld)).astype(np.float32).astype(np.float64)
        Y0 = rng.standard_normal((p.n_rows, ld)).astype(np.float32).astype(np.float64)
        Z = rng.standard_normal((p.n_rows, k)).astype(np.float32).astype(np.float64)
        R = rng.standard_normal((p.n_rows, k)).astype(np.float32).astype(np.float64)
        Xd, Yd = _dev(X, dtype), _dev(Y0, dtype)
        dot = torch.zeros(1, dtype=torch.float64, device="cuda:0")
        H.spmm_ex(Xd[:, :k], 1.5, -0.5, Yd[:, :k], gamma=0.25, Z=_dev(Z, dtype), R=_dev(R, dtype), dot_out=dot,
                  precision=prec)
        got = Yd.cpu().numpy().astype(np.float64)
        ref, scale = forward_ref(p, v, X[:, :k], 1.5, -0.5, Y0[:, :k])
        ref = ref + 0.25 * Z
        scale = scale + 0.25 * np.abs(Z)
        check_elementwise(got[:, :k], ref, scale, 1e-5)
        assert np.array_equal(got[:, k:], Y0[:, k:])          # columns beyond k untouched
        dref = float(np.sum(R * got[:, :k]))
        assert abs(dot.item() - dref) <= 1e-6 * float(np.sum(np.abs(R * got[:, :k])))

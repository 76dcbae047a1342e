"""GPU parity of the mixed-precision block products against the FP64 oracle.

Per result (Frobenius) the split modes TF32X3 and BF16X2 and the FP32 mode
must stay within 1e-5 of the FP64 oracle. Element by element the bound is
1e-4 * (|H| |X|): a single product of a bf16 hi+lo pair can be off by about
2^-16 of |h x| and FP32 accumulation over a ~300-term row adds up to
~300 * 2^-24 in the worst case, so 1e-5 per element is not guaranteed.
Single-pass TF32 (11-bit values) is expected to exceed 1e-5 and is only
checked against its own 2^-10-scale bound.
"""
import numpy as np
import pytest
import torch

import synthetic as syn
from _parity import TOL_F64, TOL_MIXED, adjoint_ref, check_elementwise, forward_ref, rel_fro

pytestmark = pytest.mark.gpu

MODES = ["f32", "tf32x3", "bf16x2"]


def _handle(pat, vals, dtype=torch.float64):
    from paper_2609_04397_gb300 import VBCSR
    return VBCSR.from_pattern(pat, vals, dtype, "cuda:0")


def _dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dtype)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("k", [1, 3, 8, 16, 33])
def test_mixed_forward_tiny_multispecies(mode, k):
    w = syn.tiny_multispecies(0)
    H = _handle(w.pattern, w.values)
    X = syn.normal_panel(w.pattern.n_cols, k, 0)
    Y0 = syn.normal_panel(w.pattern.n_rows, k, 1)
    for alpha, beta in ((1.0, 0.0), (2.0, -1.0)):
        Yd = _dev(Y0)
        H.spmm(_dev(X), alpha, beta, Yd, precision=mode)
        ref, scale = forward_ref(w.pattern, w.values, X, alpha, beta, Y0)
        got = Yd.cpu().numpy()
        assert rel_fro(got, ref) <= TOL_MIXED, rel_fro(got, ref)
        check_elementwise(got, ref, scale, 1e-4)


@pytest.mark.parametrize("mode", MODES)
def test_mixed_adjoint_and_shapes(mode):
    pat = syn.random_pattern(41, 37, (1, 4, 9, 13, 16, 20), 0.2, 12, empty_rows=2, unsorted=True)
    vals = syn.random_values(pat, 12)
    H = _handle(pat, vals)
    for k in (1, 8, 17):
        X = np.random.default_rng(k).standard_normal((pat.n_cols, k))
        got = H.spmm(_dev(X), precision=mode).cpu().numpy()
        ref, scale = forward_ref(pat, vals, X, 1.0, 0.0, None)
        assert rel_fro(got, ref) <= TOL_MIXED
        check_elementwise(got, ref, scale, 1e-4)
        Xa = np.random.default_rng(k + 1).standard_normal((pat.n_rows, k))
        got = H.spmm_adjoint(_dev(Xa), precision=mode).cpu().numpy()
        ref, scale = adjoint_ref(pat, vals, Xa, 1.0, 0.0, None)
        assert rel_fro(got, ref) <= TOL_MIXED
        check_elementwise(got, ref, scale, 1e-4)


@pytest.mark.parametrize("k", [1, 2, 8])
def test_single_tf32_within_its_own_bound(k):
    """k <= 2 runs the piece products on the CUDA cores, k = 8 on the tensor cores."""
    w = syn.tiny_multispecies(0)
    H = _handle(w.pattern, w.values)
    X = syn.normal_panel(w.pattern.n_cols, k, 0)
    got = H.spmm(_dev(X), precision="tf32").cpu().numpy()
    ref, scale = forward_ref(w.pattern, w.values, X, 1.0, 0.0, None)
    check_elementwise(got, ref, scale, 2.0 ** -9)
    assert rel_fro(got, ref) > 1e-6   # really ran in reduced precision


@pytest.mark.parametrize("mode", ["tf32", "tf32x3", "bf16x2"])
def test_thin_products_cuda_core_form_matches_tensor_core_form(mode):
    """At k <= 2 the tensor-core modes form the same piece products on the CUDA
    cores. Both forms hold the mode's bound."""
    pat = syn.random_pattern(40, 40, (1, 4, 9, 13, 16, 20), 0.25, 77, empty_rows=2, unsorted=True)
    vals = syn.random_values(pat, 77)
    H = _handle(pat, vals)
    X = np.random.default_rng(5).standard_normal((pat.n_cols, 3))
    ref, scale = forward_ref(pat, vals, X, 1.0, 0.0, None)
    tol = 2.0 ** -9 if mode == "tf32" else 1e-4
    Y3 = H.spmm(_dev(X), precision=mode).cpu().numpy()          # tensor cores (k = 3)
    Y2 = H.spmm(_dev(X[:, :2]), precision=mode).cpu().numpy()   # CUDA cores (k = 2)
    Y1 = H.spmm(_dev(X[:, 1:2]), precision=mode).cpu().numpy()  # CUDA cores (k = 1)
    check_elementwise(Y3, ref, scale, tol)
    check_elementwise(Y2, ref[:, :2], scale[:, :2], tol)
    check_elementwise(Y1[:, 0], ref[:, 1], scale[:, 1], tol)
    if mode != "tf32":
        assert rel_fro(Y2, ref[:, :2]) <= TOL_MIXED


@pytest.mark.parametrize("k", [8, 16, 33])
@pytest.mark.parametrize("mode", ["native", "tf32x3", "bf16x2"])
def test_fp32_operator_modes(mode, k):
    """FP32 operators in every mode, one to three column tiles (k = 8, 16, 33)."""
    pat = syn.random_pattern(30, 30, (4, 9, 13), 0.2, 9)
    vals = syn.random_values(pat, 9).astype(np.float32)
    H = _handle(pat, vals, torch.float32)
    X = np.random.default_rng(2).standard_normal((pat.n_cols, k)).astype(np.float32)
    got = H.spmm(_dev(X, torch.float32), precision=mode).cpu().numpy().astype(np.float64)
    ref, scale = forward_ref(pat, vals.astype(np.float64), X.astype(np.float64), 1.0, 0.0, None)
    assert rel_fro(got, ref) <= TOL_MIXED
    check_elementwise(got, ref, scale, 1e-4)


def test_mixed_copy_follows_set_values():
    pat = syn.random_pattern(20, 20, (4, 9), 0.3, 3)
    v1 = syn.random_values(pat, 3)
    H = _handle(pat, v1)
    X = np.random.default_rng(0).standard_normal((pat.n_cols, 4))
    H.spmm(_dev(X), precision="bf16x2")            # builds the FP32 copy
    v2 = syn.random_values(pat, 4)
    H.set_values(_dev(v2))
    got = H.spmm(_dev(X), precision="bf16x2").cpu().numpy()
    ref, _ = forward_ref(pat, v2, X, 1.0, 0.0, None)
    assert rel_fro(got, ref) <= TOL_MIXED
    # the CUDA-core form of a one-column product reads the same split copy
    H.set_values(_dev(v1))
    got = H.spmm(_dev(X[:, :1]), precision="bf16x2").cpu().numpy()
    ref, _ = forward_ref(pat, v1, X[:, :1], 1.0, 0.0, None)
    assert rel_fro(got, ref) <= TOL_MIXED


@pytest.mark.parametrize("mode", ["tf32", "tf32x3", "bf16x2"])
@pytest.mark.parametrize("k", [1, 8, 16, 40])
def test_staged_forward_kernel_matches_plain(mode, k):
    """The shared-memory-staged tensor-core forward kernel computes the same
    products as the plain one, incl. wide panels that span several stages and
    rows of every height. At k <= 2 both run the same CUDA-core piece products
    and agree bit for bit; at k >= 3 the plain forward of an FP64 operator is
    the pipelined kernel (bf16 planes, or FP32 operands, through a
    shared-memory ring), which feeds each MMA the same virtual columns in
    another slot order, so there the two agree to FP32 rounding of the
    accumulation."""
    pat = syn.random_pattern(45, 45, (1, 4, 9, 13, 16, 20, 70), 0.2, 40 + k, empty_rows=3, unsorted=True)
    vals = syn.random_values(pat, 40 + k)
    H = _handle(pat, vals)
    X = _dev(np.random.default_rng(k).standard_normal((pat.n_cols, k)))
    Y0 = _dev(np.random.default_rng(k + 1).standard_normal((pat.n_rows, k)))
    Yp = Y0.clone()
    H.spmm(X, 2.0, -1.0, Yp, precision=mode)
    H.set_schedule("bucketed", mma_staged=True)
    Ys = Y0.clone()
    H.spmm(X, 2.0, -1.0, Ys, precision=mode)
    if k >= 3:
        _, scale = forward_ref(pat, np.abs(vals), np.abs(X.cpu().numpy()), 2.0, 1.0, np.abs(Y0.cpu().numpy()))
        check_elementwise(Yp.cpu().numpy(), Ys.cpu().numpy().astype(np.float64), scale,
                          1e-6 if mode == "bf16x2" else 1e-5)
    else:
        assert torch.equal(Yp, Ys)
    if mode != "tf32":
        ref, scale = forward_ref(pat, vals, X.cpu().numpy(), 2.0, -1.0, Y0.cpu().numpy())
        assert rel_fro(Ys.cpu().numpy(), ref) <= TOL_MIXED


def test_autotune_picks_a_tensor_core_variant():
    w = syn.tiny_multispecies(0)
    H = _handle(w.pattern, w.values)
    t = H.autotune(8, precision="bf16x2")
    assert isinstance(t["mma_staged"], bool)
    X = syn.normal_panel(w.pattern.n_cols, 8, 0)
    got = H.spmm(_dev(X), precision="bf16x2").cpu().numpy()
    ref, _ = forward_ref(w.pattern, w.values, X, 1.0, 0.0, None)
    assert rel_fro(got, ref) <= TOL_MIXED


@pytest.mark.parametrize("mode", ["tf32", "tf32x3", "bf16x2"])
@pytest.mark.parametrize("staged", [False, True])
def test_tensor_core_products_exact_on_small_integers(mode, staged):
    """Small-integer values and X make every piece product and partial sum
    exact in FP32, so the tensor-core result in FP64 must equal the oracle bit
    for bit: at alpha = 1, at alpha = 3, at alpha = 0.1 (not an FP32 number)
    and with beta = -1. Zero blocks give exactly zero rows."""
    pat = syn.random_pattern(37, 37, (4, 9, 13, 16), 0.3, 5, empty_rows=3)
    rng = np.random.default_rng(5)
    vals = rng.integers(-4, 5, pat.nnz).astype(np.float64)
    vals[: pat.nnz // 7] = 0.0
    H = _handle(pat, vals)
    H.set_schedule("persistent", mma_staged=staged)
    for k in (8, 17, 32):
        X = rng.integers(-4, 5, (pat.n_cols, k)).astype(np.float64)
        Y0 = rng.integers(-8, 9, (pat.n_rows, k)).astype(np.float64)
        for alpha, beta in ((1.0, 0.0), (3.0, 0.0), (0.1, 0.0), (2.0, -1.0)):
            Yd = _dev(Y0)
            H.spmm(_dev(X), alpha, beta, Yd, precision=mode)
            ref, _ = forward_ref(pat, vals, X, alpha, beta, Y0)
            np.testing.assert_array_equal(Yd.cpu().numpy(), ref)


@pytest.mark.parametrize("k", [8, 13, 32, 40])
def test_fp32_value_ring_matches_direct_reads(k):
    """The per-lane-column CUDA-core forward kernel on FP32 values or
    double-FP32 pairs reads them through a shared-memory ring at k >= 8
    (default) or directly (schedule flag): the same arithmetic in the same
    order, so the results agree bit for bit, for an FP32 operator and for the
    F32 and DF32 modes of an FP64 operator, on rows taller than 16 and panels
    wider than one staged window. The pipelined FP32 kernel of the persistent
    launch meets the FP32 bound against the oracle on the same cases."""
    pat = syn.random_pattern(12, 14, (3, 9, 20, 60), 0.5, 31 + k, empty_rows=1)
    vals = syn.random_values(pat, 31)
    X = np.random.default_rng(k).standard_normal((pat.n_cols, k))
    for dtype, prec in ((torch.float32, "native"), (torch.float64, "f32"), (torch.float64, "df32")):
        H = _handle(pat, vals.astype(np.float32) if dtype == torch.float32 else vals, dtype)
        Xd = _dev(X, dtype)
        ref, scale = forward_ref(pat, vals, X, 1.0, 0.0, None)
        for sch in ("persistent", "bucketed"):
            H.set_schedule(sch, pipelined_f32=False)
            got_ring = H.spmm(Xd, precision=prec).cpu().numpy()
            H.set_schedule(sch, value_ring=False, pipelined_f32=False)
            got_direct = H.spmm(Xd, precision=prec).cpu().numpy()
            np.testing.assert_array_equal(got_ring, got_direct)
            check_elementwise(got_ring.astype(np.float64), ref, scale, TOL_F64 if prec == "df32" else 1e-4)
        # the persistent default on FP32 values: the pipelined kernel (another summation order)
        H.set_schedule("persistent")
        got_pipe = H.spmm(Xd, precision=prec).cpu().numpy()
        check_elementwise(got_pipe.astype(np.float64), ref, scale, TOL_F64 if prec == "df32" else 1e-4)



@pytest.mark.parametrize("mode", ["tf32", "tf32x3", "bf16x2"])
@pytest.mark.parametrize("k", [4, 16, 20])
def test_recurrence_with_converted_vectors_matches_per_step_conversion(mode, k):
    """In the tensor-core modes the Chebyshev recurrence keeps each t_n also
    in the form the kernel reads (written by the previous step's epilogue)
    instead of converting it before every product. The same recurrence run
    step by step through vbcsr_spmm_ex (which converts X at every call) gives
    the same moments bit for bit; the doubling moments stay within 1e-5 of
    the oracle's."""
    import oracle
    w = syn.tiny_multispecies(0)
    c, d = oracle.cheb_scale(w.pattern, w.values)
    vt = oracle.shift_scale_values(w.pattern, w.values, c, d)
    H = _handle(w.pattern, vt)
    Rn = syn.rademacher_panel(w.pattern.n_rows, k, 0)
    R = _dev(Rn)
    M = 40
    fused = H.chebyshev(R, M, precision=mode)[0]
    mu = torch.empty(M, dtype=torch.float64, device="cuda:0")
    mu[0] = (R * R).sum() / R.numel()
    T = [R.clone(), torch.empty_like(R)]
    H.spmm_ex(R, 1.0, 0.0, T[1], R=R, dot_out=mu[1:2], precision=mode)
    for n in range(1, M - 1):
        # t_{n+1} = 2 H~ t_n - t_{n-1}, overwriting t_{n-1}
        H.spmm_ex(T[n & 1], 2.0, -1.0, T[(n + 1) & 1], R=R, dot_out=mu[n + 1:n + 2], precision=mode)
    mu[1:] *= 1.0 / R.numel()          # the library multiplies the raw dot by 1 / (N k)
    assert torch.equal(fused[1:], mu[1:]), (fused - mu).abs().max().item()
    ref = oracle.chebyshev_moments(w.pattern, vt, Rn, M)
    tol = 1e-5 if mode != "tf32" else 1e-2
    assert np.abs(fused.cpu().numpy() - ref).max() <= tol
    kpm = H.kpm_moments(R, M, precision=mode).cpu().numpy()
    assert np.abs(kpm - ref).max() <= tol



@pytest.mark.parametrize("k", [3, 8, 16, 20, 32])
def test_pipelined_kernels_on_ragged_shapes(k):
    """The pipelined tensor-core (BF16X2, TF32X3, TF32 of an FP64 operator),
    FP32 (FP32 operator, F32 mode) and double-FP32 (DF32 mode) forward
    kernels on an operator with empty block rows (items without
    columns), rows taller than 16 (several items per block row) and rows wider
    than 512 virtual columns (several shared-memory windows per item), with
    alpha, beta, gamma Z and the fused dot: every element within the mode's
    bound of the oracle, the dot equal to the oracle's sum of R * Y within
    the same bound, and alpha = 0 reading no product."""
    pat = syn.random_pattern(14, 40, (3, 9, 20, 60), 0.6, 70 + k, empty_rows=2)
    vals = syn.random_values(pat, 71)
    assert int(pat.row_bsize.max()) > 16
    kw = [int(pat.col_bsize[pat.block_col_idx[pat.block_row_ptr[i]:pat.block_row_ptr[i + 1]]].sum())
          for i in range(len(pat.row_bsize))]
    assert max(kw) > 512 and min(kw) == 0
    rng = np.random.default_rng(k)
    X = rng.standard_normal((pat.n_cols, k))
    Y0 = rng.standard_normal((pat.n_rows, k))
    Zn = rng.standard_normal((pat.n_rows, k))
    Rn = rng.standard_normal((pat.n_rows, k))
    cases = [(torch.float64, "bf16x2", 1e-4), (torch.float64, "tf32x3", 1e-4), (torch.float64, "tf32", 2.0 ** -9)]
    if k >= 8:
        cases += [(torch.float32, "native", 1e-4), (torch.float64, "f32", 1e-4), (torch.float64, "df32", TOL_F64)]
    for dtype, prec, tol in cases:
        H = _handle(pat, vals.astype(np.float32) if dtype == torch.float32 else vals, dtype)
        for alpha, beta, gamma in ((1.0, 0.0, 0.0), (2.0, -1.0, 0.5), (0.0, 1.5, 0.0)):
            Yd = _dev(Y0, dtype)
            dot = torch.zeros(1, dtype=torch.float64, device="cuda:0")
            H.spmm_ex(_dev(X, dtype), alpha, beta, Yd, gamma=gamma, Z=_dev(Zn, dtype), R=_dev(Rn, dtype),
                      dot_out=dot, precision=prec)
            ref, scale = forward_ref(pat, vals, X, alpha, beta, Y0)
            ref = ref + gamma * Zn
            got = Yd.cpu().numpy().astype(np.float64)
            check_elementwise(got, ref, scale + abs(gamma) * np.abs(Zn), tol)
            rdot = float(np.sum(Rn * ref))
            bound = tol * float(np.sum(np.abs(Rn) * (scale + abs(gamma) * np.abs(Zn))))
            assert abs(dot.item() - rdot) <= bound, (prec, alpha, dot.item(), rdot)

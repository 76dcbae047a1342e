"""VBCSR oracle: plain, slow, obviously correct CPU reference of the hot path.

TEST INFRASTRUCTURE ONLY. Only the tests, the repository smoke check and the
benchmark's CPU-baseline / reference legs may import this package; the
product library never does, and this package imports nothing from it.

Contents, each following the passage it cites:

* ``spmm``          Y = alpha H X + beta Y, scalar-expanded FP64 loop (C),
                    Sec. III.B "Matrix multiplication"
* ``spmm_adjoint``  Y = alpha H^T X + beta Y, Eq. (1) with real values (C)
* ``sddmm``         D_ij = alpha A_i B_j^T + beta D_ij on the stored pattern (C);
                    the gradient of H X with respect to the stored values
* ``to_dense``      dense assembly of the block operator (Sec. II.A)
* ``chebyshev_moments`` / ``moment_loss_grad``  the kernel-polynomial-method
                    recurrence of Sec. V (t_{n+1} = 2 H~ t_n - t_{n-1}) and the
                    reverse-mode gradient of L = sum_n mu_n^2
* ``kpm_moments_doubling`` / ``kpm_dos`` / ``kpm_gap``  the DOS pipeline of
                    Sec. V (moments, damped DOS, the gap read off it)
* ``spgemm``        the thresholded block product, Eqs. (2)-(3)
* ``kspace_blocks`` / ``kspace_dense``  a periodic operator sampled in
                    reciprocal space, Eq. (4); ``spmm_complex`` /
                    ``spmm_adjoint_complex`` its block products (Eq. 1 with a
                    conjugate transpose)

A pattern argument is any object with the attributes ``row_bsize``,
``col_bsize``, ``block_row_ptr`` and ``block_col_idx`` (numpy arrays).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vbcsr_oracle.c")
_SO = os.path.join(_HERE, "_lib", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile vbcsr_oracle.c with gcc into oracle/_lib/liboracle.so."""
    with _lock:
        if (not force and os.path.exists(_SO)
                and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
            return _SO
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                        "-ffp-contract=off", _SRC, "-o", tmp], check=True)
        os.replace(tmp, _SO)
        return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        i64, p, d, i32 = ctypes.c_int64, ctypes.c_void_p, ctypes.c_double, ctypes.c_int
        L.oracle_spmm.argtypes = [i64, i64, p, p, p, p, p, i64, d, p, i64, d, p, i64, i64, i64, i32]
        L.oracle_spmm_adjoint.argtypes = [i64, i64, p, p, p, p, p, i64, d, p, i64, d, p, i64]
        L.oracle_sddmm.argtypes = [i64, i64, p, p, p, p, i64, d, p, i64, p, i64, d, p, i32]
        L.oracle_gershgorin.argtypes = [i64, i64, p, p, p, p, p, p]
        for f in (L.oracle_spmm, L.oracle_spmm_adjoint, L.oracle_sddmm, L.oracle_gershgorin):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _c(a, dt):
    a = np.ascontiguousarray(a, dtype=dt)
    return a, a.ctypes.data


def _pat(pat):
    rb, prb = _c(pat.row_bsize, np.int32)
    cb, pcb = _c(pat.col_bsize, np.int32)
    rp, prp = _c(pat.block_row_ptr, np.int64)
    ci, pci = _c(pat.block_col_idx, np.int32)
    return (rb, cb, rp, ci), (len(rb), len(cb), prb, pcb, prp, pci)


def n_rows(pat) -> int:
    return int(np.asarray(pat.row_bsize, np.int64).sum())


def n_cols(pat) -> int:
    return int(np.asarray(pat.col_bsize, np.int64).sum())


# ----------------------------------------------------------------------------
# the three products (C loops)


def spmm(pat, values, X, alpha=1.0, beta=0.0, Y=None, row_range=None, nthreads=1):
    """Y = alpha H X + beta Y (Sec. III.B). X is [n_cols, k] (row-major, any
    leading dimension via a 2-D view). Returns Y as a new [n_rows, k] array
    (Y is copied first when beta != 0). row_range=(b0, b1) restricts the
    computation to block rows b0..b1-1; other rows of the result are then
    whatever Y held (zero if Y is None)."""
    keep, args = _pat(pat)
    X = np.ascontiguousarray(X, dtype=np.float64)
    k = X.shape[1]
    out = np.zeros((n_rows(pat), k)) if Y is None else np.array(Y, dtype=np.float64, order="C", copy=True)
    v, pv = _c(values, np.float64)
    b0, b1 = (0, len(keep[0])) if row_range is None else row_range
    rc = _load().oracle_spmm(*args, pv, k, float(alpha), X.ctypes.data, k, float(beta),
                             out.ctypes.data, k, int(b0), int(b1), int(nthreads))
    if rc:
        raise MemoryError("oracle_spmm")
    return out


def spmm_adjoint(pat, values, X, alpha=1.0, beta=0.0, Y=None):
    """Y = alpha H^T X + beta Y (Eq. 1, real values). X is [n_rows, k]."""
    keep, args = _pat(pat)
    X = np.ascontiguousarray(X, dtype=np.float64)
    k = X.shape[1]
    out = np.zeros((n_cols(pat), k)) if Y is None else np.array(Y, dtype=np.float64, order="C", copy=True)
    v, pv = _c(values, np.float64)
    rc = _load().oracle_spmm_adjoint(*args, pv, k, float(alpha), X.ctypes.data, k, float(beta),
                                     out.ctypes.data, k)
    if rc:
        raise MemoryError("oracle_spmm_adjoint")
    return out


def sddmm(pat, A, B, alpha=1.0, beta=0.0, D=None, nthreads=1):
    """D_ij[p,q] = alpha sum_c A[r_i+p, c] B[c_j+q, c] + beta D_ij[p,q] on the
    stored blocks, in packed value order. A is [n_rows, k], B is [n_cols, k]."""
    keep, args = _pat(pat)
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    k = A.shape[1]
    assert B.shape[1] == k
    rb, cb, rp, ci = keep
    nnz = int((rb[np.repeat(np.arange(len(rb)), np.diff(rp))].astype(np.int64) * cb[ci]).sum())
    out = np.zeros(nnz) if D is None else np.array(D, dtype=np.float64, copy=True)
    rc = _load().oracle_sddmm(*args, k, float(alpha), A.ctypes.data, k, B.ctypes.data, k,
                              float(beta), out.ctypes.data, int(nthreads))
    if rc:
        raise MemoryError("oracle_sddmm")
    return out


# ----------------------------------------------------------------------------
# dense assembly (Sec. II.A: block (i, j) is a dense b_i x b_j matrix at
# scalar rows r_i.. and columns c_j..)


def to_dense(pat, values) -> np.ndarray:
    rb = np.asarray(pat.row_bsize, np.int64)
    cb = np.asarray(pat.col_bsize, np.int64)
    r = np.concatenate([[0], np.cumsum(rb)])
    c = np.concatenate([[0], np.cumsum(cb)])
    H = np.zeros((r[-1], c[-1]))
    off = 0
    for i in range(len(rb)):
        for b in range(pat.block_row_ptr[i], pat.block_row_ptr[i + 1]):
            j = int(pat.block_col_idx[b])
            n = int(rb[i] * cb[j])
            H[r[i]:r[i + 1], c[j]:c[j + 1]] += np.asarray(values[off:off + n]).reshape(rb[i], cb[j])
            off += n
    return H


# ----------------------------------------------------------------------------
# kernel polynomial method (Sec. V): Chebyshev recurrence and moments


def gershgorin_bounds(pat, values):
    """(E_min, E_max) from Gershgorin discs over scalar rows: every eigenvalue
    of a square H lies in [min_p (H_pp - R_p), max_p (H_pp + R_p)], R_p the
    off-diagonal absolute row sum (C loop, O(n_rows) memory)."""
    keep, args = _pat(pat)
    v, pv = _c(values, np.float64)
    out = np.zeros(2)
    if _load().oracle_gershgorin(*args, pv, out.ctypes.data):
        raise MemoryError("oracle_gershgorin")
    return float(out[0]), float(out[1])


def cheb_scale(pat, values, pad: float = 1.01):
    """Centre c and half-width d so that H~ = (H - c I) / d has its spectrum
    inside [-1, 1]: c = (E+ + E-)/2, d = pad * (E+ - E-)/2."""
    lo, hi = gershgorin_bounds(pat, values)
    return 0.5 * (hi + lo), pad * 0.5 * (hi - lo)


def shift_scale_values(pat, values, c, d, inplace: bool = False) -> np.ndarray:
    """Packed values of H~ = (H - c I) / d (c subtracted on the scalar diagonal);
    with inplace=True the float64 array `values` itself is overwritten."""
    rb = np.asarray(pat.row_bsize, np.int64)
    cb = np.asarray(pat.col_bsize, np.int64)
    r = np.concatenate([[0], np.cumsum(rb)])
    cc = np.concatenate([[0], np.cumsum(cb)])
    rows = np.repeat(np.arange(len(rb)), np.diff(pat.block_row_ptr))
    cols = np.asarray(pat.block_col_idx, np.int64)
    off = np.concatenate([[0], np.cumsum(rb[rows] * cb[cols])])
    out = values if inplace else np.array(values, dtype=np.float64, copy=True)
    for b in np.nonzero((r[rows] < cc[cols] + cb[cols]) & (cc[cols] < r[rows] + rb[rows]))[0]:
        i, j = rows[b], cols[b]
        for p in range(rb[i]):
            q = r[i] + p - cc[j]
            if 0 <= q < cb[j]:
                out[off[b] + p * cb[j] + q] -= c
    np.divide(out, d, out=out)
    return out


def chebyshev_vectors(pat, values_t, R, n_moments):
    """t_0 = R, t_1 = H~ R, t_{n+1} = 2 H~ t_n - t_{n-1}; returns [t_0 .. t_{M-1}]."""
    t = [np.array(R, dtype=np.float64)]
    if n_moments > 1:
        t.append(spmm(pat, values_t, t[0]))
    for n in range(1, n_moments - 1):
        t.append(spmm(pat, values_t, t[n], alpha=2.0, beta=-1.0, Y=t[n - 1]))
    return t


def chebyshev_moments(pat, values_t, R, n_moments, nthreads=1) -> np.ndarray:
    """mu_n = <R, t_n> / (N * n_vec) for n = 0 .. n_moments - 1 (stochastic
    trace estimate of T_n(H~) / N, kernel polynomial method). Keeps only the
    last two vectors of the recurrence."""
    R = np.asarray(R, dtype=np.float64)
    mu = [float(np.sum(R * R))]
    if n_moments > 1:
        prev, cur = R, spmm(pat, values_t, R, nthreads=nthreads)
        mu.append(float(np.sum(R * cur)))
        for n in range(1, n_moments - 1):
            prev, cur = cur, spmm(pat, values_t, cur, alpha=2.0, beta=-1.0, Y=prev, nthreads=nthreads)
            mu.append(float(np.sum(R * cur)))
    return np.array(mu) / R.size


def moment_loss(pat, values_t, R, n_moments) -> float:
    """L = sum_n mu_n^2."""
    return float(np.sum(chebyshev_moments(pat, values_t, R, n_moments) ** 2))


def moment_loss_grad(pat, values_t, R, n_moments) -> np.ndarray:
    """dL/dH~ on the stored values, by the reverse recurrence:

    g_n = dL/dt_n (direct) = 2 mu_n R / (N n_vec),
    lam_n = g_n + 2 H~^T lam_{n+1} - lam_{n+2}   (lam_M = lam_{M+1} = 0, n >= 1),
    dL/dH~ = lam_1 t_0^T + sum_{n=1}^{M-2} 2 lam_{n+1} t_n^T   (on the pattern).
    """
    R = np.asarray(R, dtype=np.float64)
    M = n_moments
    t = chebyshev_vectors(pat, values_t, R, M)
    mu = np.array([float(np.sum(R * tn)) for tn in t]) / R.size
    g = [2.0 * mu[n] * R / R.size for n in range(M)]
    lam = [None] * (M + 2)
    zero = np.zeros_like(R)
    lam[M] = zero
    lam[M + 1] = zero
    for n in range(M - 1, 0, -1):
        lam[n] = g[n] + spmm_adjoint(pat, values_t, lam[n + 1], alpha=2.0) - lam[n + 2]
    grad = np.zeros(len(np.asarray(values_t)))
    if M > 1:
        grad += sddmm(pat, lam[1], t[0])
    for n in range(1, M - 1):
        grad += sddmm(pat, lam[n + 1], t[n], alpha=2.0)
    return grad


# ----------------------------------------------------------------------------
# kernel polynomial method: moments by the doubling identities, Jackson
# damping, DOS reconstruction (Sec. V; Weisse, Wellein, Alvermann & Fehske,
# Rev. Mod. Phys. 78, 275 (2006), Sec. II)


def kpm_moments_doubling(pat, values_t, R, n_moments, nthreads=1) -> np.ndarray:
    """mu_0 .. mu_{M-1} of a symmetric H~ from t_0 .. t_{ceil(M/2)} using
    T_{2n} = 2 T_n^2 - T_0 and T_{2n+1} = 2 T_{n+1} T_n - T_1:
    mu_{2n} = 2 <t_n, t_n> / (N k) - mu_0,  mu_{2n+1} = 2 <t_{n+1}, t_n> / (N k) - mu_1."""
    R = np.asarray(R, dtype=np.float64)
    s = 1.0 / R.size
    mu = np.zeros(n_moments)
    mu[0] = np.sum(R * R) * s
    if n_moments == 1:
        return mu
    t_prev, t_cur = R, spmm(pat, values_t, R, nthreads=nthreads)      # t_0, t_1
    mu[1] = np.sum(t_cur * R) * s
    n = 1                                                               # t_cur = t_n
    while True:
        if 2 * n < n_moments:
            mu[2 * n] = 2.0 * np.sum(t_cur * t_cur) * s - mu[0]
        if 2 * n + 1 >= n_moments:
            break
        t_next = spmm(pat, values_t, t_cur, alpha=2.0, beta=-1.0, Y=t_prev, nthreads=nthreads)
        mu[2 * n + 1] = 2.0 * np.sum(t_next * t_cur) * s - mu[1]
        t_prev, t_cur = t_cur, t_next
        n += 1
    return mu


def jackson_kernel(n_moments) -> np.ndarray:
    """Jackson damping factors g_n, n = 0 .. M-1 (M = n_moments):
    g_n = [(M - n + 1) cos(pi n / (M + 1)) + sin(pi n / (M + 1)) cot(pi / (M + 1))] / (M + 1)."""
    M = n_moments
    n = np.arange(M, dtype=np.float64)
    q = np.pi / (M + 1)
    return ((M - n + 1) * np.cos(q * n) + np.sin(q * n) / np.tan(q)) / (M + 1)


def kpm_dos(mu, x, kernel="jackson") -> np.ndarray:
    """rho(x) = [g_0 mu_0 + 2 sum_{n>=1} g_n mu_n T_n(x)] / (pi sqrt(1 - x^2)),
    x in (-1, 1) (the scaled energy), T_n(x) = cos(n arccos x)."""
    mu = np.asarray(mu, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    g = jackson_kernel(len(mu)) if kernel == "jackson" else np.ones(len(mu))
    th = np.arccos(x)
    acc = g[0] * mu[0] * np.ones_like(x)
    for n in range(1, len(mu)):
        acc += 2.0 * g[n] * mu[n] * np.cos(n * th)
    return acc / (np.pi * np.sqrt(1.0 - x * x))


def kpm_gap(energies, dos, reference, threshold):
    """Band gap read off a density of states (Sec. V reads the gaps of the InP
    particles off their KPM DOS with a threshold criterion; the threshold is
    an argument here). With i0 the grid point nearest `reference` (the first
    one on a tie), walk left and right from i0 while the next point's DOS is
    below `threshold` (NaN is not below); returns (energies[lo], energies[hi])
    of that run, or None when dos[i0] itself is not below the threshold."""
    E = [float(e) for e in energies]
    D = [float(v) for v in dos]
    i0 = 0
    for j in range(1, len(E)):
        if abs(E[j] - reference) < abs(E[i0] - reference):
            i0 = j
    if not (D[i0] < threshold):
        return None
    lo = i0
    while lo - 1 >= 0 and D[lo - 1] < threshold:
        lo -= 1
    hi = i0
    while hi + 1 < len(E) and D[hi + 1] < threshold:
        hi += 1
    return E[lo], E[hi]


# ----------------------------------------------------------------------------
# thresholded block sparse product (Sec. III.B, Eqs. 2-3)


def block_norms(pat, values) -> np.ndarray:
    """Frobenius norm of every stored block (packed order)."""
    off = pat.value_offset() if hasattr(pat, "value_offset") else None
    rb = np.asarray(pat.row_bsize, np.int64)
    cb = np.asarray(pat.col_bsize, np.int64)
    rows = np.repeat(np.arange(len(rb)), np.diff(pat.block_row_ptr))
    sizes = rb[rows] * cb[np.asarray(pat.block_col_idx, np.int64)]
    if off is None:
        off = np.concatenate([[0], np.cumsum(sizes)])
    v = np.asarray(values, np.float64)
    return np.sqrt(np.add.reduceat(v * v, off[:-1])) if len(sizes) else np.zeros(0)


def spgemm(patA, valsA, patB, valsB, eps):
    """C = A B on block patterns (patA's column blocks are patB's row blocks).
    Symbolic stage: a candidate block (i, j) is kept when the bound
    sum_k ||A_ik|| ||B_kj|| (Eq. 3) is >= eps; numeric stage: C_ij = sum_k A_ik B_kj
    (Eq. 2) over every k with both blocks stored; final filter: blocks with
    ||C_ij|| < eps are removed. Returns (row_bsize, col_bsize, block_row_ptr,
    block_col_idx, values) with columns sorted inside each row; norms are
    Frobenius norms."""
    nA = block_norms(patA, valsA)
    nB = block_norms(patB, valsB)
    ra = np.asarray(patA.row_bsize, np.int64)
    kb = np.asarray(patB.row_bsize, np.int64)
    cb = np.asarray(patB.col_bsize, np.int64)
    offA = np.concatenate([[0], np.cumsum(ra[np.repeat(np.arange(len(ra)), np.diff(patA.block_row_ptr))]
                                          * np.asarray(patA.col_bsize, np.int64)[np.asarray(patA.block_col_idx)])])
    offB = np.concatenate([[0], np.cumsum(kb[np.repeat(np.arange(len(kb)), np.diff(patB.block_row_ptr))]
                                          * cb[np.asarray(patB.block_col_idx)])])
    ptr, cols, vals = [0], [], []
    for i in range(len(ra)):
        bound = {}
        for a in range(patA.block_row_ptr[i], patA.block_row_ptr[i + 1]):
            k = int(patA.block_col_idx[a])
            for b in range(patB.block_row_ptr[k], patB.block_row_ptr[k + 1]):
                j = int(patB.block_col_idx[b])
                bound[j] = bound.get(j, 0.0) + nA[a] * nB[b]
        kept = sorted(j for j, bd in bound.items() if bd >= eps)
        for j in kept:
            Cij = np.zeros((ra[i], cb[j]))
            for a in range(patA.block_row_ptr[i], patA.block_row_ptr[i + 1]):
                k = int(patA.block_col_idx[a])
                Aik = np.asarray(valsA[offA[a]:offA[a + 1]]).reshape(ra[i], kb[k])
                for b in range(patB.block_row_ptr[k], patB.block_row_ptr[k + 1]):
                    if int(patB.block_col_idx[b]) == j:
                        Bkj = np.asarray(valsB[offB[b]:offB[b + 1]]).reshape(kb[k], cb[j])
                        Cij += Aik @ Bkj
            if np.sqrt(np.sum(Cij * Cij)) >= eps:
                cols.append(j)
                vals.append(Cij.ravel())
        ptr.append(len(cols))
    return (ra.astype(np.int32), cb.astype(np.int32), np.array(ptr, np.int64), np.array(cols, np.int32),
            np.concatenate(vals) if vals else np.zeros(0))


# ----------------------------------------------------------------------------
# periodic operators in reciprocal space (Sec. III.C "Atomistic Interfaces",
# Eq. 4) and complex block products


def kspace_blocks(bsize, edge_i, edge_j, edge_R, edge_values, kfrac, tau=None):
    """O(k) on the union pattern of the edges (Eq. 4): block (i, j) is
    sum over the edges (i, j, R) of exp(-2 pi i k . s) O(R)_ij with s = R, or
    s = R + tau_j - tau_i when fractional positions tau are given. Edges are
    (i, j, R) triples with real b_i x b_j blocks packed row-major in edge order.
    Returns (row_bsize, col_bsize, block_row_ptr, block_col_idx, values) with the
    union blocks in row order, columns increasing, values complex128."""
    bs = np.asarray(bsize, np.int64)
    ei, ej = np.asarray(edge_i, np.int64), np.asarray(edge_j, np.int64)
    R = np.asarray(edge_R, np.float64).reshape(-1, 3)
    k = np.asarray(kfrac, np.float64).reshape(3)
    off = np.concatenate([[0], np.cumsum(bs[ei] * bs[ej])])
    blocks = {}
    for e in range(len(ei)):
        i, j = int(ei[e]), int(ej[e])
        s = R[e].copy()
        if tau is not None:
            t = np.asarray(tau, np.float64).reshape(-1, 3)
            s = s + t[j] - t[i]
        phase = np.exp(-2j * np.pi * float(k @ s))
        O = np.asarray(edge_values[off[e]:off[e + 1]], np.float64).reshape(bs[i], bs[j])
        blocks[(i, j)] = blocks.get((i, j), 0) + phase * O
    keys = sorted(blocks)
    ptr = np.zeros(len(bs) + 1, np.int64)
    for (i, _j) in keys:
        ptr[i + 1] += 1
    ptr = np.cumsum(ptr)
    cols = np.array([j for (_i, j) in keys], np.int32)
    vals = np.concatenate([np.asarray(blocks[key], np.complex128).ravel() for key in keys]) if keys \
        else np.zeros(0, np.complex128)
    return bs.astype(np.int32), bs.astype(np.int32), ptr, cols, vals


def kspace_dense(bsize, edge_i, edge_j, edge_R, edge_values, kfrac, tau=None) -> np.ndarray:
    """Dense O(k) (Eq. 4), each edge's phased block added straight into the
    dense matrix at scalar rows r_i.. and columns r_j.."""
    bs = np.asarray(bsize, np.int64)
    r = np.concatenate([[0], np.cumsum(bs)])
    ei, ej = np.asarray(edge_i, np.int64), np.asarray(edge_j, np.int64)
    R = np.asarray(edge_R, np.float64).reshape(-1, 3)
    k = np.asarray(kfrac, np.float64).reshape(3)
    off = np.concatenate([[0], np.cumsum(bs[ei] * bs[ej])])
    H = np.zeros((r[-1], r[-1]), np.complex128)
    for e in range(len(ei)):
        i, j = int(ei[e]), int(ej[e])
        s = R[e] if tau is None else R[e] + np.asarray(tau, np.float64).reshape(-1, 3)[j] \
            - np.asarray(tau, np.float64).reshape(-1, 3)[i]
        O = np.asarray(edge_values[off[e]:off[e + 1]], np.float64).reshape(bs[i], bs[j])
        H[r[i]:r[i + 1], r[j]:r[j + 1]] += np.exp(-2j * np.pi * float(k @ s)) * O
    return H


def _block_loop(pat, values, X, alpha, beta, Y, adjoint):
    rb = np.asarray(pat.row_bsize, np.int64)
    cb = np.asarray(pat.col_bsize, np.int64)
    r = np.concatenate([[0], np.cumsum(rb)])
    c = np.concatenate([[0], np.cumsum(cb)])
    X = np.asarray(X, np.complex128)
    n_out = c[-1] if adjoint else r[-1]
    acc = np.zeros((n_out, X.shape[1]), np.complex128)
    off = 0
    for i in range(len(rb)):
        for b in range(pat.block_row_ptr[i], pat.block_row_ptr[i + 1]):
            j = int(pat.block_col_idx[b])
            n = int(rb[i] * cb[j])
            Hij = np.asarray(values[off:off + n], np.complex128).reshape(rb[i], cb[j])
            off += n
            if adjoint:
                acc[c[j]:c[j + 1]] += Hij.conj().T @ X[r[i]:r[i + 1]]
            else:
                acc[r[i]:r[i + 1]] += Hij @ X[c[j]:c[j + 1]]
    out = alpha * acc
    if beta != 0.0 and Y is not None:
        out = out + beta * np.asarray(Y, np.complex128)
    return out


def spmm_complex(pat, values, X, alpha=1.0, beta=0.0, Y=None) -> np.ndarray:
    """Y = alpha H X + beta Y for complex blocks: Y_i += H_ij X_j block by block
    (Sec. III.B "Matrix multiplication"); beta == 0: Y is not read."""
    return _block_loop(pat, values, X, alpha, beta, Y, adjoint=False)


def spmm_adjoint_complex(pat, values, X, alpha=1.0, beta=0.0, Y=None) -> np.ndarray:
    """Y = alpha H^dagger X + beta Y: Y_j += H_ij^dagger X_i (Eq. 1), the
    dagger a conjugate transpose."""
    return _block_loop(pat, values, X, alpha, beta, Y, adjoint=True)


def gershgorin_bounds_complex(pat, values):
    """(E_min, E_max) of a complex Hermitian operator from Gershgorin discs
    over scalar rows: [min_p (Re H_pp - R_p), max_p (Re H_pp + R_p)], R_p the
    sum of the moduli |H_pq| over q != p."""
    rb = np.asarray(pat.row_bsize, np.int64)
    cb = np.asarray(pat.col_bsize, np.int64)
    r = np.concatenate([[0], np.cumsum(rb)])
    c = np.concatenate([[0], np.cumsum(cb)])
    diag = np.zeros(r[-1])
    off = np.zeros(r[-1])
    o = 0
    for i in range(len(rb)):
        for b in range(pat.block_row_ptr[i], pat.block_row_ptr[i + 1]):
            j = int(pat.block_col_idx[b])
            blk = np.asarray(values[o:o + rb[i] * cb[j]], np.complex128).reshape(rb[i], cb[j])
            o += rb[i] * cb[j]
            for p in range(rb[i]):
                for q in range(cb[j]):
                    if r[i] + p == c[j] + q:
                        diag[r[i] + p] += blk[p, q].real
                    else:
                        off[r[i] + p] += abs(blk[p, q])
    return float(np.min(diag - off)), float(np.max(diag + off))


def shift_scale_values_complex(pat, values, c, d) -> np.ndarray:
    """Packed values of H~ = (H - c I) / d for a complex operator: c subtracted
    from the scalar diagonal, every entry divided by d."""
    out = np.array(values, dtype=np.complex128, copy=True)
    re = shift_scale_values(pat, out.real.copy(), c, d)
    return re + 1j * (out.imag / d)


def chebyshev_moments_complex(pat, values_t, R, n_moments) -> np.ndarray:
    """mu_n = Re <R, t_n> / (N * n_vec), t_0 = R, t_1 = H~ R,
    t_{n+1} = 2 H~ t_n - t_{n-1}, for a complex (Hermitian) H~ and complex R."""
    R = np.asarray(R, dtype=np.complex128)
    mu = [float(np.vdot(R, R).real)]
    if n_moments > 1:
        prev, cur = R, spmm_complex(pat, values_t, R)
        mu.append(float(np.vdot(R, cur).real))
        for n in range(1, n_moments - 1):
            prev, cur = cur, spmm_complex(pat, values_t, cur, 2.0, -1.0, prev)
            mu.append(float(np.vdot(R, cur).real))
    return np.array(mu) / R.size

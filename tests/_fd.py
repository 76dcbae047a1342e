"""Central finite differences of the Chebyshev moment loss, evaluated with
the oracle and without cancellation (test helper)."""
import numpy as np

import oracle


def central_difference(pat, vals, R, M, i, h, nthreads=1):
    """(L(v + h e_i) - L(v - h e_i)) / (2h) for L = sum_n mu_n^2, evaluated
    without cancellation: with H+- = H~(v +- h e_i), d_n = t_n^+ - t_n^- obeys
      d_0 = 0,  d_1 = (H+ - H-) R,  d_{n+1} = 2 H+ d_n + 2 (H+ - H-) t_n^- - d_{n-1},
    and (H+ - H-) is 2h at the stored entry i, so L+ - L- = sum_n dmu_n (2 mu_n^- + dmu_n)
    with dmu_n = <R, d_n> / (N k)."""
    off = pat.value_offset()
    b = int(np.searchsorted(off, i, side="right") - 1)
    row_blk = int(np.searchsorted(pat.block_row_ptr, b, side="right") - 1)
    j = int(pat.block_col_idx[b])
    bj = int(pat.col_bsize[j])
    p, q = divmod(int(i - off[b]), bj)
    r = int(np.sum(pat.row_bsize[:row_blk])) + p
    c = int(np.sum(pat.col_bsize[:j])) + q
    vp, vm = vals.copy(), vals.copy()
    vp[i] += h
    vm[i] -= h

    def e_times(X):              # (H+ - H-) X
        out = np.zeros((pat.n_rows, X.shape[1]))
        out[r] = 2.0 * h * X[c]
        return out

    s = 1.0 / R.size
    tm_prev, tm = R, oracle.spmm(pat, vm, R, nthreads=nthreads)
    d_prev, d = np.zeros_like(R), e_times(R)
    mu_m = [np.sum(R * R) * s, np.sum(R * tm) * s]
    dmu = [0.0, np.sum(R * d) * s]
    for n in range(1, M - 1):
        d_next = oracle.spmm(pat, vp, d, alpha=2.0, beta=-1.0, Y=d_prev, nthreads=nthreads) + 2.0 * e_times(tm)
        tm_next = oracle.spmm(pat, vm, tm, alpha=2.0, beta=-1.0, Y=tm_prev, nthreads=nthreads)
        d_prev, d, tm_prev, tm = d, d_next, tm, tm_next
        mu_m.append(np.sum(R * tm) * s)
        dmu.append(np.sum(R * d) * s)
    mu_m, dmu = np.array(mu_m), np.array(dmu)
    return float(np.sum(dmu * (2.0 * mu_m + dmu)) / (2.0 * h))

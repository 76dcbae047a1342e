"""Writes zincblende_1m_moments.json: FP64 oracle Chebyshev moments of the
~1e6-atom zinc-blende workload (the precision form at scale).

Recipe: synthetic.zincblende(1_000_000, seed=0) (cation b = 13, anion b = 9,
third neighbour shell plus self, entries exp(-r/2 A) N(0,1), symmetric);
c, d from the oracle's Gershgorin bounds (c = (E+ + E-)/2, d = 1.01 (E+ - E-)/2);
H~ = (H - c I)/d; 16 Rademacher vectors synthetic.rademacher_panel(N, 16, 0);
moments mu_0 .. mu_50 of t_0 = R, t_1 = H~ R, t_{n+1} = 2 H~ t_n - t_{n-1}.
Calls only the oracle and the input generator. Needs ~35 GB of host memory.

    python tests/golden/make_zincblende_1m_moments.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synthetic as syn  # noqa: E402

N_ATOMS, K, M = 1_000_000, 16, 51


def main():
    t0 = time.time()
    w = syn.zincblende(N_ATOMS, seed=0)
    pat = w.pattern
    threads = os.cpu_count() or 1
    lo, hi = oracle.gershgorin_bounds(pat, w.values)
    c, d = 0.5 * (hi + lo), 1.01 * 0.5 * (hi - lo)
    vt = oracle.shift_scale_values(pat, w.values, c, d, inplace=True)
    R = syn.rademacher_panel(pat.n_rows, K, 0)
    mu = oracle.chebyshev_moments(pat, vt, R, M, nthreads=threads)
    out = {
        "source": "FP64 oracle (oracle.chebyshev_moments) on synthetic.zincblende(1_000_000, seed=0); "
                  "written by tests/golden/make_zincblende_1m_moments.py",
        "n_atoms": int(pat.n_brows), "n_rows": int(pat.n_rows), "nblk": int(pat.nblk), "nnz": int(pat.nnz),
        "gershgorin": [lo, hi], "c": c, "d": d, "k": K, "n_moments": M, "R": "rademacher_panel(n_rows, 16, 0)",
        "moments": [float(x) for x in mu], "oracle_threads": threads, "seconds": time.time() - t0,
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "zincblende_1m_moments.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k != "moments"}))


if __name__ == "__main__":
    main()

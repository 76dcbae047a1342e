"""The precision form at scale: the ~1e6-atom zinc-blende operator (~3.3e9
stored entries, 26.7 GB in FP64), a 50-step Chebyshev recurrence with 16
Rademacher vectors, block products in FP64, double-FP32, TF32X3 and BF16X2
with the recurrence and the moments in FP64; every moment against the FP64
oracle's (tests/golden/zincblende_1m_moments.json, written by
tests/golden/make_zincblende_1m_moments.py)."""
import json
import os
import time

import numpy as np
import pytest
import torch

import synthetic as syn

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "zincblende_1m_moments.json")
TOL = {"native": 1e-12, "df32": 1e-12, "tf32x3": 1e-5, "bf16x2": 1e-5}


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="golden moments not generated")
def test_zincblende_1m_chebyshev_precision_form():
    from paper_2609_04397_gb300 import VBCSR
    with open(GOLDEN) as f:
        g = json.load(f)
    w = syn.zincblende(g["n_atoms_target"] if "n_atoms_target" in g else 1_000_000, seed=0)
    pat = w.pattern
    assert (pat.n_brows, pat.n_rows, pat.nnz) == (g["n_atoms"], g["n_rows"], g["nnz"])
    H = VBCSR.from_pattern(pat, w.values, torch.float64, "cuda:0")
    del w
    lo, hi = H.gershgorin()
    assert abs(lo - g["gershgorin"][0]) <= 1e-12 * abs(g["gershgorin"][0])
    assert abs(hi - g["gershgorin"][1]) <= 1e-12 * abs(g["gershgorin"][1])
    H.shift_scale(g["c"], g["d"])
    R = torch.from_numpy(syn.rademacher_panel(g["n_rows"], g["k"], 0)).cuda()
    ref = np.array(g["moments"])
    report = {}
    for prec in ("native", "df32", "tf32x3", "bf16x2"):
        H.chebyshev(R, 3, precision=prec)            # first use builds the copies the mode needs
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mom, _ = H.chebyshev(R, g["n_moments"], precision=prec)
        e1.record()
        torch.cuda.synchronize()
        err = np.abs(mom.cpu().numpy() - ref) / abs(ref[0])
        report[prec] = {"ms": e0.elapsed_time(e1), "max_moment_err": float(err.max())}
    base = report["native"]["ms"]
    for prec, r in report.items():
        r["speedup_vs_f64"] = base / r["ms"]
    print("zincblende 1e6 precision form:", json.dumps(report))
    for prec, r in report.items():
        assert r["max_moment_err"] <= TOL[prec], (prec, r)
    H.check()

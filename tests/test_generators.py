"""Invariants of the seeded synthetic inputs (no product arithmetic here)."""
import json
import os

import numpy as np

import oracle
import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _blocks(pat):
    rows = pat.block_rows()
    return set(zip(rows.tolist(), pat.block_col_idx.tolist()))


def test_tiny_multispecies_shape():
    w = syn.tiny_multispecies(0)
    p = w.pattern
    assert p.n_brows == 200 and p.n_rows == 100 * 4 + 100 * 9 == 1300
    assert sorted(np.unique(p.row_bsize).tolist()) == [4, 9]
    blocks = _blocks(p)
    assert all((j, i) in blocks for (i, j) in blocks)          # symmetric pattern
    assert all((i, i) in blocks for i in range(p.n_brows))     # diagonal present
    # columns sorted inside each row
    for i in range(p.n_brows):
        c = p.block_col_idx[p.block_row_ptr[i]:p.block_row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_symmetric_values_are_symmetric():
    w = syn.tiny_multispecies(0)
    H = oracle.to_dense(w.pattern, w.values)
    assert np.array_equal(H, H.T)


def test_generator_is_deterministic_and_seeded():
    a = syn.tiny_multispecies(0)
    b = syn.tiny_multispecies(0)
    c = syn.tiny_multispecies(1)
    assert np.array_equal(a.values, b.values)
    assert not np.array_equal(a.pattern.block_col_idx[:50], c.pattern.block_col_idx[:50]) or \
        not np.array_equal(a.values[:50], c.values[:50])
    x1 = syn.normal_panel(100, 3, 0)
    x2 = syn.normal_panel(100, 5, 0, ld=5)
    assert np.array_equal(x1, syn.normal_panel(100, 3, 0))
    assert abs(x2.mean()) < 0.2 and abs(x2.std() - 1.0) < 0.1
    r = syn.rademacher_panel(1000, 4, 0)
    assert set(np.unique(r).tolist()) == {-1.0, 1.0}


def test_zincblende_shells_and_bulk_rows():
    with open(os.path.join(GOLDEN, "zincblende_shells.json")) as f:
        g = json.load(f)
    w = syn.zincblende(3000, with_values=False)
    p, sys = w.pattern, w.system
    a = g["a"]
    counts = np.diff(p.block_row_ptr)
    assert counts.max() == g["blocks_per_bulk_row"]
    # an interior atom (far from the surface) has exactly the textbook shells
    r = np.linalg.norm(sys.pos, axis=1)
    i = int(np.argmin(r))
    nb = p.block_col_idx[p.block_row_ptr[i]:p.block_row_ptr[i + 1]]
    d = np.sort(np.linalg.norm(sys.pos[nb] - sys.pos[i], axis=1))[1:] / a
    expect = np.concatenate([np.full(s["count"], s["r_over_a"]) for s in g["shells"]])
    assert np.allclose(d, expect, atol=1e-9)
    # cation b=13, anion b=9 and the per-block distances are consistent
    assert set(np.unique(p.row_bsize).tolist()) == {9, 13}
    assert np.all(p.block_dist <= g["cutoff_over_a"] * a)


def test_morton_order_is_local():
    w = syn.zincblende(3000, with_values=False)
    pos = w.system.pos
    step = np.linalg.norm(np.diff(pos, axis=0), axis=1)
    rand = np.linalg.norm(np.diff(pos[np.random.default_rng(0).permutation(len(pos))], axis=0), axis=1)
    # consecutive atoms sit within the third neighbour shell (5.4 A) in most cases
    assert np.median(step) < 5.4 < np.median(rand) / 4


def test_batched_offsets_and_independence():
    w = syn.batched_uneven(n_structs=6, n_min=50, n_max=120, seed=3)
    p = w.pattern
    offs = w.struct_brow_offsets
    assert offs[0] == 0 and offs[-1] == p.n_brows and len(offs) == 7
    rows = p.block_rows()
    s_row = np.searchsorted(offs, rows, side="right") - 1
    s_col = np.searchsorted(offs, p.block_col_idx, side="right") - 1
    assert np.array_equal(s_row, s_col)                       # block diagonal
    assert set(np.unique(p.row_bsize).tolist()) <= {4, 9, 13}


def test_amorphous_min_separation_small():
    w = syn.amorphous(n=800, side=60.0 * (800 / 20000) ** (1 / 3), with_values=False)
    sys = w.system
    from scipy.spatial import cKDTree
    d, _ = cKDTree(np.mod(sys.pos, sys.box), boxsize=sys.box).query(np.mod(sys.pos, sys.box), k=2)
    assert d[:, 1].min() >= 1.8 - 1e-12
    counts = np.bincount(sys.bsize)
    assert counts[4] == 320 and counts[9] == 320 and counts[13] == 160

"""The seeded synthetic workloads: operators, input panels and random vectors.

Five families stand in for the paper's workloads (Sec. IV atom-like
geometric graphs; Sec. V zinc-blende nanoparticles):

* ``tiny_multispecies``   200 atoms, b in {4, 9}, periodic 16 A cube, 5 A cutoff
* ``zincblende``          spherical zinc-blende cluster, cation b=13, anion b=9,
                          blocks to the third neighbour shell plus self
* ``amorphous``           random sequential placement, b in {4, 9, 13} 40/40/20
* ``batched_uneven``      many independent periodic structures of uneven size
* ``domain``              ~500 MiB scalar / uniform-block / variable-block graphs

Values follow a symmetric construction (H_ji = H_ij^T). All random numbers
come from the counter-based generator in gen.c; nothing here computes a
sparse product.
"""
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import _native
from .structures import (AtomSystem, BlockPattern, amorphous_cube, block_diagonal,
                         morton_order, neighbor_pattern, random_cube, reorder,
                         zincblende_sphere)

# stream ids for the counter-based generator
STREAM_VALUES = 1
STREAM_X = 2
STREAM_RADEMACHER = 3
STREAM_GENERIC = 4

ZB_A = 5.87                       # zinc-blende lattice constant (Angstrom)
ZB_CUTOFF = 0.9146 * ZB_A         # between the 3rd (sqrt(11)/4 a) and 4th (a) shells


def stream_key(seed: int, stream: int) -> int:
    return int(_native.lib().syn_stream_key(seed, stream))


# ----------------------------------------------------------------------------
# values and panels


def symmetric_values(pat: BlockPattern, scale: np.ndarray, seed: int = 0) -> np.ndarray:
    """Packed values of a symmetric operator on a square, symmetric pattern
    (see syn_symmetric_values in gen.c for the exact recipe)."""
    assert pat.n_brows == pat.n_bcols and np.array_equal(pat.row_bsize, pat.col_bsize)
    off = pat.value_offset()
    out = np.empty(int(off[-1]), dtype=np.float64)
    scale = np.ascontiguousarray(scale, dtype=np.float64)
    rc = _native.lib().syn_symmetric_values(
        stream_key(seed, STREAM_VALUES), pat.n_brows, _native.ptr(pat.row_bsize),
        _native.ptr(pat.block_row_ptr), _native.ptr(pat.block_col_idx),
        _native.ptr(off), _native.ptr(scale), _native.ptr(out))
    if rc != 0:
        raise ValueError("block sizes must lie in [1, 32]")
    return out


def random_values(pat: BlockPattern, seed: int = 0) -> np.ndarray:
    """Independent N(0,1) entries for every stored value (no symmetry)."""
    n = pat.nnz
    out = np.empty(n, dtype=np.float64)
    cnt = np.arange(n, dtype=np.uint64)
    _native.lib().syn_normal_at(stream_key(seed, STREAM_GENERIC), n, _native.ptr(cnt), _native.ptr(out))
    return out


def normal_panel(nrows: int, ncols: int, seed: int = 0, stream: int = STREAM_X,
                 ld: Optional[int] = None) -> np.ndarray:
    """Row-major [nrows, ld] panel whose first ncols columns are N(0,1)."""
    ld = ncols if ld is None else ld
    out = np.zeros((nrows, ld), dtype=np.float64)
    _native.lib().syn_normal_panel(stream_key(seed, stream), nrows, ncols, ld, _native.ptr(out))
    return out


def rademacher_panel(nrows: int, ncols: int, seed: int = 0) -> np.ndarray:
    """Row-major [nrows, ncols] panel of +1/-1 entries."""
    out = np.empty((nrows, ncols), dtype=np.float64)
    _native.lib().syn_sign_panel(stream_key(seed, STREAM_RADEMACHER), nrows, ncols, ncols,
                                 _native.ptr(out))
    return out


def nnz_row_scale(pat: BlockPattern) -> np.ndarray:
    """Per-block scale (n_i n_j)^(-1/4), n_i = scalar entries in a row of atom i,
    so that a row of H has variance about 1 (entries N(0,1)/sqrt(nnz_row))."""
    rows = pat.block_rows()
    n_i = np.bincount(rows, weights=pat.col_bsize[pat.block_col_idx].astype(np.float64),
                      minlength=pat.n_brows)
    return (n_i[rows] * n_i[pat.block_col_idx]) ** -0.25


def decay_scale(pat: BlockPattern, length: float = 2.0) -> np.ndarray:
    """Per-block scale exp(-r / length), r the atom distance in Angstrom."""
    return np.exp(-pat.block_dist / length)


# ----------------------------------------------------------------------------
# workloads


@dataclass
class Workload:
    name: str
    pattern: BlockPattern
    values: Optional[np.ndarray]
    system: Optional[AtomSystem] = None
    struct_brow_offsets: Optional[np.ndarray] = None   # batched only: [n_structs + 1]
    struct_bcol_offsets: Optional[np.ndarray] = None


def _ordered(sys: AtomSystem) -> AtomSystem:
    return reorder(sys, morton_order(sys.pos, 1.0))


def tiny_multispecies(seed: int = 0, with_values: bool = True) -> Workload:
    """200 atoms uniformly random in a periodic 16 A cube, b=4 and b=9 50/50,
    5 A cutoff plus self; entries N(0,1)/sqrt(nnz_row), symmetric."""
    sys = _ordered(random_cube(200, 16.0, (4, 9), (0.5, 0.5), seed))
    pat = neighbor_pattern(sys, 5.0)
    vals = symmetric_values(pat, nnz_row_scale(pat), seed) if with_values else None
    return Workload("tiny_multispecies_200", pat, vals, sys)


def zincblende(n_target: int = 50_000, seed: int = 0, with_values: bool = True) -> Workload:
    """Spherical zinc-blende cluster (a = 5.87 A, cation b=13, anion b=9),
    blocks to the third neighbour shell plus self, entries exp(-r/2A) N(0,1),
    symmetric, open boundary."""
    sys = _ordered(zincblende_sphere(n_target, ZB_A, 13, 9))
    pat = neighbor_pattern(sys, ZB_CUTOFF)
    vals = symmetric_values(pat, decay_scale(pat, 2.0), seed) if with_values else None
    return Workload(f"zincblende_{len(sys.bsize)}", pat, vals, sys)


def amorphous(n: int = 20_000, side: float = 60.0, seed: int = 0,
              with_values: bool = True) -> Workload:
    """Random amorphous system: n atoms in a periodic cube, minimum separation
    1.8 A, b in {4, 9, 13} at 40/40/20 %, 4.5 A cutoff; entries as
    tiny_multispecies."""
    sys = _ordered(amorphous_cube(n, side, 1.8, (4, 9, 13), (0.4, 0.4, 0.2), seed))
    pat = neighbor_pattern(sys, 4.5)
    vals = symmetric_values(pat, nnz_row_scale(pat), seed) if with_values else None
    return Workload(f"amorphous_{n}", pat, vals, sys)


def batched_uneven(n_structs: int = 256, n_min: int = 50, n_max: int = 2000,
                   density: float = 0.0488, cutoff: float = 5.0, seed: int = 0,
                   with_values: bool = True) -> Workload:
    """Independent periodic structures with log-uniform atom counts in
    [n_min, n_max], b in {4, 9, 13} in equal thirds, cube side
    (n / density)^(1/3), 5 A cutoff; concatenated block-diagonally."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=n_structs))).astype(int)
    pats: List[BlockPattern] = []
    for s, n in enumerate(sizes):
        side = (n / density) ** (1.0 / 3.0)
        sys = _ordered(random_cube(int(n), side, (4, 9, 13), (1 / 3, 1 / 3, 1 / 3), seed * 100_003 + s + 1))
        pats.append(neighbor_pattern(sys, cutoff))
    pat = block_diagonal(pats)
    boffs = np.zeros(n_structs + 1, np.int64)
    np.cumsum([p.n_brows for p in pats], out=boffs[1:])
    vals = symmetric_values(pat, nnz_row_scale(pat), seed) if with_values else None
    wl = Workload(f"batched_{n_structs}", pat, vals, None, boffs, boffs.copy())
    wl.parts = pats
    return wl


def domain(kind: str, target_bytes: float = 500 * 2 ** 20, seed: int = 0) -> Workload:
    """Atom-like periodic geometric graphs sized to ~target_bytes of stored
    values and indices, in the three structural domains of the paper's kernel
    benchmark (Sec. IV): 'csr' (every b = 1), 'bsr' (every b = 8) and 'vbcsr'
    (b uniform at random in [9, 20]). Cube at density 0.0488 / A^3 with a
    5 A cutoff plus self (~26 blocks per row); entries as tiny_multispecies."""
    rng = np.random.default_rng(seed)
    dens, cutoff, deg = 0.0488, 5.0, 26.6
    # stored bytes per block row: blocks x (values + one column index)
    per_row = {"csr": deg * (8 + 4), "bsr": deg * (64 * 8 + 4), "vbcsr": deg * (14.5 ** 2 * 8 + 4)}[kind]
    n = int(target_bytes / per_row)
    side = (n / dens) ** (1.0 / 3.0)
    pos = rng.uniform(0.0, side, size=(n, 3))
    if kind == "csr":
        b = np.ones(n, np.int32)
    elif kind == "bsr":
        b = np.full(n, 8, np.int32)
    else:
        b = rng.integers(9, 21, size=n).astype(np.int32)
    sys = _ordered(AtomSystem(pos, b, side))
    pat = neighbor_pattern(sys, cutoff)
    vals = symmetric_values(pat, nnz_row_scale(pat), seed)
    return Workload(f"domain_{kind}_{n}", pat, vals, sys)


# ----------------------------------------------------------------------------
# periodic operators as lattice images


@dataclass
class PeriodicWorkload:
    name: str
    bsize: np.ndarray            # int32 [n_atoms]
    edge_i: np.ndarray           # int32 [n_edges]
    edge_j: np.ndarray
    edge_R: np.ndarray           # int32 [n_edges, 3]
    edge_dist: np.ndarray        # float64 [n_edges], Angstrom
    edge_values: np.ndarray      # float64, the edges' blocks packed row-major in edge order
    tau: np.ndarray              # float64 [n_atoms, 3], fractional positions in the box


def image_values(bsize, edge_i, edge_j, edge_R, edge_dist, seed: int = 0, length: float = 2.0) -> np.ndarray:
    """Real blocks of a symmetric periodic operator: O(j, i, -R) = O(i, j, R)^T
    (so that every O(k) is Hermitian), entries exp(-r / length) N(0, 1), the
    (i, i, 0) blocks (G + G^T) / sqrt(2); drawn from the counter-based generator
    keyed by the canonical orientation of each edge."""
    bs = np.asarray(bsize, np.int64)
    ei, ej = np.asarray(edge_i, np.int64), np.asarray(edge_j, np.int64)
    eR = np.asarray(edge_R, np.int64).reshape(-1, 3)
    fwd = np.column_stack([ei, ej, eR])
    rev = np.column_stack([ej, ei, -eR])
    # canonical orientation: the lexicographically smaller of the edge and its mirror
    use_rev = np.zeros(len(ei), bool)
    for c in range(5):
        undecided = ~use_rev & np.all(fwd[:, :c] == rev[:, :c], axis=1)
        use_rev |= undecided & (rev[:, c] < fwd[:, c])
    canon = np.where(use_rev[:, None], rev, fwd)
    keys, cid = np.unique(canon, axis=0, return_inverse=True)
    cid = cid.reshape(-1)
    ca, cb = bs[keys[:, 0]], bs[keys[:, 1]]
    coff = np.concatenate([[0], np.cumsum(ca * cb)])
    G = np.empty(int(coff[-1]), np.float64)
    cnt = np.arange(len(G), dtype=np.uint64)
    _native.lib().syn_normal_at(stream_key(seed, STREAM_GENERIC), len(G), _native.ptr(cnt), _native.ptr(G))
    out = []
    for e in range(len(ei)):
        c = cid[e]
        blk = G[coff[c]:coff[c + 1]].reshape(ca[c], cb[c])
        if keys[c, 0] == keys[c, 1] and not keys[c, 2:].any():
            blk = (blk + blk.T) / np.sqrt(2.0)          # (i, i, 0): its own mirror
        elif use_rev[e]:
            blk = blk.T
        out.append((np.exp(-edge_dist[e] / length) * blk).ravel())
    return np.concatenate(out) if out else np.zeros(0)


def zincblende_crystal(n_cells: int = 2, seed: int = 0) -> PeriodicWorkload:
    """Periodic zinc-blende crystal (a = 5.87 A, cation b = 13, anion b = 9)
    of n_cells^3 conventional cells, images to the third neighbour shell plus
    self (the nanoparticle's cutoff), entries exp(-r/2 A) N(0,1), symmetric."""
    from .structures import periodic_images, zincblende_cell
    sys = zincblende_cell(n_cells, ZB_A)
    ei, ej, eR, ed = periodic_images(sys, ZB_CUTOFF)
    vals = image_values(sys.bsize, ei, ej, eR, ed, seed)
    return PeriodicWorkload(f"zincblende_crystal_{len(sys.bsize)}", sys.bsize, ei, ej, eR, ed, vals,
                            np.mod(sys.pos, sys.box) / sys.box)

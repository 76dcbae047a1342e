"""Seeded synthetic atom systems and their block-sparse patterns.

Each atom carries b orbitals (its block size); an interaction block (i, j)
exists for i == j and for every pair within the cutoff. The systems stand in
for the paper's workloads (atom-like periodic geometric graphs with a finite
cutoff, Sec. IV; zinc-blende nanoparticles, Sec. V); none of the paper's own
structures or tight-binding parameters are used.

Nothing here performs the sparse product: this module only draws inputs.
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np
from scipy.spatial import cKDTree


@dataclass
class BlockPattern:
    """A variable-block CSR pattern (Sec. II.A): block row i has height
    row_bsize[i]; its stored blocks are block_col_idx[block_row_ptr[i]:
    block_row_ptr[i+1]]; block (i, j) is row_bsize[i] x col_bsize[j]."""
    row_bsize: np.ndarray       # int32 [n_brows]
    col_bsize: np.ndarray       # int32 [n_bcols]
    block_row_ptr: np.ndarray   # int64 [n_brows + 1]
    block_col_idx: np.ndarray   # int32 [nblk]
    block_dist: Optional[np.ndarray] = None   # float64 [nblk], atom distance (Angstrom)
    meta: dict = field(default_factory=dict)

    def __post_init__(self):
        self.row_bsize = np.ascontiguousarray(self.row_bsize, dtype=np.int32)
        self.col_bsize = np.ascontiguousarray(self.col_bsize, dtype=np.int32)
        self.block_row_ptr = np.ascontiguousarray(self.block_row_ptr, dtype=np.int64)
        self.block_col_idx = np.ascontiguousarray(self.block_col_idx, dtype=np.int32)

    @property
    def n_brows(self) -> int:
        return len(self.row_bsize)

    @property
    def n_bcols(self) -> int:
        return len(self.col_bsize)

    @property
    def nblk(self) -> int:
        return len(self.block_col_idx)

    @property
    def n_rows(self) -> int:
        return int(self.row_bsize.sum())

    @property
    def n_cols(self) -> int:
        return int(self.col_bsize.sum())

    def block_rows(self) -> np.ndarray:
        """Block-row index of every stored block."""
        return np.repeat(np.arange(self.n_brows, dtype=np.int64),
                         np.diff(self.block_row_ptr))

    def block_sizes(self) -> np.ndarray:
        """Number of entries b_i * b_j of every stored block."""
        return (self.row_bsize[self.block_rows()].astype(np.int64)
                * self.col_bsize[self.block_col_idx].astype(np.int64))

    def value_offset(self) -> np.ndarray:
        """int64 [nblk + 1]: start of each block in the packed value array."""
        off = np.zeros(self.nblk + 1, dtype=np.int64)
        np.cumsum(self.block_sizes(), out=off[1:])
        return off

    @property
    def nnz(self) -> int:
        return int(self.block_sizes().sum())


@dataclass
class AtomSystem:
    pos: np.ndarray             # float64 [n, 3], Angstrom
    bsize: np.ndarray           # int32 [n]
    box: Optional[float]        # periodic cube side, or None (open boundary)


# ----------------------------------------------------------------------------
# geometry


def _spread_bits(v: np.ndarray) -> np.ndarray:
    """Insert two zero bits between the low 21 bits of v (Morton encoding)."""
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_order(pos: np.ndarray, grid: float = 1.0) -> np.ndarray:
    """Permutation that sorts atoms along a Z-order curve on a `grid` lattice
    (ties keep their original order)."""
    q = np.floor((pos - pos.min(axis=0)) / grid).astype(np.int64)
    code = (_spread_bits(q[:, 0]) | (_spread_bits(q[:, 1]) << np.uint64(1))
            | (_spread_bits(q[:, 2]) << np.uint64(2)))
    return np.argsort(code, kind="stable")


def reorder(sys: AtomSystem, perm: np.ndarray) -> AtomSystem:
    return AtomSystem(sys.pos[perm].copy(), sys.bsize[perm].copy(), sys.box)


def _species(rng, n: int, sizes, fractions) -> np.ndarray:
    counts = [int(round(f * n)) for f in fractions]
    counts[-1] = n - sum(counts[:-1])
    b = np.concatenate([np.full(c, s, dtype=np.int32) for s, c in zip(sizes, counts)])
    return b[rng.permutation(n)]


def random_cube(n: int, side: float, sizes, fractions, seed: int) -> AtomSystem:
    """n atoms uniformly at random in a periodic cube; species counts fixed by
    `fractions`, assigned in random order."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, side, size=(n, 3))
    b = _species(rng, n, sizes, fractions)
    return AtomSystem(pos, b, side)


def amorphous_cube(n: int, side: float, min_sep: float, sizes, fractions,
                   seed: int, batch: int = 4096) -> AtomSystem:
    """Random sequential placement in a periodic cube: candidates uniform at
    random, each kept only if it is at least `min_sep` from every kept atom
    (candidates are taken in draw order)."""
    rng = np.random.default_rng(seed)
    kept = np.empty((0, 3))
    while len(kept) < n:
        cand = rng.uniform(0.0, side, size=(batch, 3))
        if len(kept):
            d, _ = cKDTree(kept, boxsize=side).query(cand, k=1)
            cand = cand[d >= min_sep]
        if len(cand) > 1:
            pairs = cKDTree(cand, boxsize=side).query_pairs(min_sep, output_type="ndarray")
            keep = np.ones(len(cand), dtype=bool)
            if len(pairs):
                pairs = np.sort(pairs, axis=1)
                order = np.lexsort((pairs[:, 0], pairs[:, 1]))
                for a, b in pairs[order]:
                    if keep[a]:
                        keep[b] = False
            cand = cand[keep]
        kept = np.concatenate([kept, cand[: n - len(kept)]])
    b = _species(rng, n, sizes, fractions)
    return AtomSystem(kept, b, side)


def zincblende_sphere(n_target: int, a: float = 5.87, b_cation: int = 13,
                      b_anion: int = 9) -> AtomSystem:
    """Spherical zinc-blende cluster centred on a cation: cations on the fcc
    sites of a cubic cell of side a, anions shifted by (a/4)(1,1,1); the radius
    is chosen so that the sphere holds about n_target atoms (8 atoms per a^3)."""
    radius = (3.0 * n_target * a ** 3 / (4.0 * np.pi * 8.0)) ** (1.0 / 3.0)
    m = int(np.ceil(radius / a)) + 1
    r = np.arange(-m, m + 1, dtype=np.float64)
    cells = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3) * a
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]]) * a
    cat = (cells[:, None, :] + fcc[None]).reshape(-1, 3)
    ani = cat + a / 4.0
    pos = np.concatenate([cat, ani])
    bs = np.concatenate([np.full(len(cat), b_cation, np.int32),
                         np.full(len(ani), b_anion, np.int32)])
    inside = np.einsum("ij,ij->i", pos, pos) <= radius * radius
    return AtomSystem(pos[inside], bs[inside], None)


# ----------------------------------------------------------------------------
# patterns


def neighbor_pattern(sys: AtomSystem, cutoff: float) -> BlockPattern:
    """Block pattern with a diagonal block for every atom and a block (i, j)
    and (j, i) for every pair closer than `cutoff` (minimum image when the box
    is periodic; the box must exceed 2 * cutoff so a pair has one image).
    Columns are sorted inside each block row."""
    n = len(sys.bsize)
    if sys.box is not None:
        assert sys.box > 2.0 * cutoff, "box must exceed twice the cutoff"
        tree = cKDTree(np.mod(sys.pos, sys.box), boxsize=sys.box)
    else:
        tree = cKDTree(sys.pos)
    pairs = tree.query_pairs(cutoff, output_type="ndarray").astype(np.int64)
    d = sys.pos[pairs[:, 1]] - sys.pos[pairs[:, 0]]
    if sys.box is not None:
        d -= sys.box * np.round(d / sys.box)
    dist = np.sqrt(np.einsum("ij,ij->i", d, d))
    ii = np.concatenate([np.arange(n), pairs[:, 0], pairs[:, 1]])
    jj = np.concatenate([np.arange(n), pairs[:, 1], pairs[:, 0]])
    dd = np.concatenate([np.zeros(n), dist, dist])
    order = np.lexsort((jj, ii))
    ii, jj, dd = ii[order], jj[order], dd[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(ii, minlength=n), out=row_ptr[1:])
    return BlockPattern(sys.bsize, sys.bsize, row_ptr, jj.astype(np.int32), dd)


def block_diagonal(patterns) -> BlockPattern:
    """Concatenate independent patterns into one block-diagonal pattern."""
    rbs = np.concatenate([p.row_bsize for p in patterns])
    cbs = np.concatenate([p.col_bsize for p in patterns])
    ptrs, cols, dists = [np.zeros(1, np.int64)], [], []
    boff, coff = 0, 0
    for p in patterns:
        ptrs.append(p.block_row_ptr[1:] + boff)
        cols.append(p.block_col_idx.astype(np.int64) + coff)
        if p.block_dist is not None:
            dists.append(p.block_dist)
        boff += p.nblk
        coff += p.n_bcols
    dist = np.concatenate(dists) if len(dists) == len(patterns) else None
    return BlockPattern(rbs, cbs, np.concatenate(ptrs), np.concatenate(cols).astype(np.int32), dist)


def random_pattern(n_brows: int, n_bcols: int, sizes, density: float, seed: int,
                   empty_rows: int = 0, unsorted: bool = False) -> BlockPattern:
    """Random rectangular pattern: each (i, j) present with probability
    `density`; `empty_rows` randomly chosen block rows are left empty; with
    `unsorted` the columns inside a row are shuffled."""
    rng = np.random.default_rng(seed)
    rbs = rng.choice(np.asarray(sizes, np.int32), size=n_brows)
    cbs = rng.choice(np.asarray(sizes, np.int32), size=n_bcols)
    mask = rng.random((n_brows, n_bcols)) < density
    if empty_rows:
        mask[rng.choice(n_brows, size=min(empty_rows, n_brows), replace=False)] = False
    ptr = np.zeros(n_brows + 1, dtype=np.int64)
    np.cumsum(mask.sum(axis=1), out=ptr[1:])
    cols = []
    for i in range(n_brows):
        c = np.nonzero(mask[i])[0]
        if unsorted:
            c = rng.permutation(c)
        cols.append(c)
    col = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    return BlockPattern(rbs, cbs, ptr, col.astype(np.int32))


# ----------------------------------------------------------------------------
# periodic crystals as lattice images


def zincblende_cell(n_cells: int, a: float = 5.87, b_cation: int = 13, b_anion: int = 9) -> AtomSystem:
    """Periodic zinc-blende crystal of n_cells^3 conventional cubic cells (8
    atoms each: cations on the fcc sites, anions shifted by (a/4)(1,1,1)); the
    periodic box has side n_cells * a."""
    r = np.arange(n_cells, dtype=np.float64)
    cells = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3) * a
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]]) * a
    cat = (cells[:, None, :] + fcc[None]).reshape(-1, 3)
    ani = cat + a / 4.0
    pos = np.concatenate([cat, ani])
    bs = np.concatenate([np.full(len(cat), b_cation, np.int32), np.full(len(ani), b_anion, np.int32)])
    return AtomSystem(pos, bs, n_cells * a)


def periodic_images(sys: AtomSystem, cutoff: float):
    """Edges (i, j, R) of a periodic system: every atom pair and lattice
    translation R (integer multiples of the box) with |pos_j + R box - pos_i| <
    cutoff, including (i, i, 0). Returns (edge_i, edge_j, edge_R [n, 3],
    distance), sorted by (i, j, R). A box wider than twice the cutoff gives at
    most one R per pair (minimum image); a smaller one is enumerated."""
    assert sys.box is not None
    n, L = len(sys.bsize), float(sys.box)
    pos = np.mod(sys.pos, L)
    if L > 2.0 * cutoff:
        tree = cKDTree(pos, boxsize=L)
        pairs = tree.query_pairs(cutoff, output_type="ndarray").astype(np.int64)
        d = pos[pairs[:, 1]] - pos[pairs[:, 0]]
        R = -np.round(d / L).astype(np.int64)           # image of j nearest to i
        dd = d + R * L
        dist = np.sqrt(np.einsum("ij,ij->i", dd, dd))
        ei = np.concatenate([np.arange(n), pairs[:, 0], pairs[:, 1]])
        ej = np.concatenate([np.arange(n), pairs[:, 1], pairs[:, 0]])
        eR = np.concatenate([np.zeros((n, 3), np.int64), R, -R])
        ed = np.concatenate([np.zeros(n), dist, dist])
    else:
        m = int(np.ceil(cutoff / L))
        tree = cKDTree(pos)
        parts = []
        for rx in range(-m, m + 1):
            for ry in range(-m, m + 1):
                for rz in range(-m, m + 1):
                    R = np.array([rx, ry, rz], np.int64)
                    other = cKDTree(pos + R * L)
                    for i, js in enumerate(tree.query_ball_tree(other, cutoff)):
                        for j in js:
                            dv = pos[j] + R * L - pos[i]
                            parts.append((i, j, rx, ry, rz, float(np.sqrt(dv @ dv))))
        arr = np.array(parts, dtype=np.float64)
        ei, ej = arr[:, 0].astype(np.int64), arr[:, 1].astype(np.int64)
        eR, ed = arr[:, 2:5].astype(np.int64), arr[:, 5]
    order = np.lexsort((eR[:, 2], eR[:, 1], eR[:, 0], ej, ei))
    return (ei[order].astype(np.int32), ej[order].astype(np.int32), eR[order].astype(np.int32), ed[order])

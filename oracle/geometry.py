"""Level / region / stream geometry (oracle; test infrastructure only).

Sec. IV (multilevel hierarchy): level l keeps the points of level l-1 with even
indices along every axis, so the stride doubles per level; the decomposition
produces L levels and level L-1 is the coarse representation.

Reading used here (the paper's Algorithm 1/2 loop bounds are off by one):
levels 0 .. L-2 are predicted, with stride s = 2^l; level L-1 is the 2^(L-1)
grid, stored raw (predicted by zero).

Regions (Sec. IV "per-region interpolation", Sec. V-C "3(L-1)+1 regions"):
with pass order pi over the d active axes, region r (1-based) of level l is the
set of points that are odd multiples of s along pi(r), multiples of 2s along
pi(r+1..d) and multiples of s along pi(1..r-1).  Fig. 4's 500x500x250 region 3
of a 500^3 field is the last region, compacted along the last (fastest) axis.

Streams: a stream is a list of lattices (arithmetic progressions in every
axis), concatenated; each lattice is stored in row-major order with every row
(fixed k0, k1) padded with zeros to a multiple of 32 elements, so that one
32-bit plane word never straddles two rows.  The paper does not fix a byte
layout (it stores each region in its own buffer, Sec. VI-C); this padded
row-major layout is the reading used by both the oracle and the library.
"""
from dataclasses import dataclass, field
from typing import List, Tuple

WORD = 32           # elements per plane word
SEG_ELEMS = 4096    # elements per sign segment (generic encoding)


def active_axes(shape3):
    """Axes that are refined.  2-D fields are stored as (1, n1, n2)."""
    return tuple(a for a in range(3) if shape3[a] > 1)


def auto_levels(shape3):
    """L = max(1, floor(log2(min_active n - 1))): the coarsest grid keeps at
    least 3 points per active axis."""
    m = min(shape3[a] for a in active_axes(shape3))
    L = 0
    while (1 << (L + 1)) <= m - 1:
        L += 1
    return max(1, L)


def max_levels(shape3):
    """Largest L whose coarsest grid keeps at least 2 points per active axis."""
    m = min(shape3[a] for a in active_axes(shape3))
    L = 1
    while (1 << L) <= m - 1:
        L += 1
    return L


def count_from(n, start, step):
    """Number of indices start, start+step, ... below n."""
    if n - 1 < start:
        return 0
    return (n - 1 - start) // step + 1


@dataclass(frozen=True)
class Lattice:
    start: Tuple[int, int, int]
    step: Tuple[int, int, int]
    count: Tuple[int, int, int]

    @property
    def n_real(self):
        return self.count[0] * self.count[1] * self.count[2]

    @property
    def row_pad(self):
        return -(-self.count[2] // WORD) * WORD

    @property
    def n_pad(self):
        return self.count[0] * self.count[1] * self.row_pad

    def slices(self):
        return tuple(slice(st, st + sp * (c - 1) + 1, sp) if c > 0 else slice(0, 0)
                     for st, sp, c in zip(self.start, self.step, self.count))

    def empty(self):
        return self.n_real == 0


def region_lattice(shape3, level, order, r):
    """Region r (1-based) of level ``level`` with pass order ``order``."""
    s = 1 << level
    start, step, count = [0, 0, 0], [1, 1, 1], [1, 1, 1]
    a = order[r - 1]
    start[a], step[a], count[a] = s, 2 * s, count_from(shape3[a], s, 2 * s)
    for b in order[r:]:
        start[b], step[b], count[b] = 0, 2 * s, count_from(shape3[b], 0, 2 * s)
    for b in order[:r - 1]:
        start[b], step[b], count[b] = 0, s, count_from(shape3[b], 0, s)
    return Lattice(tuple(start), tuple(step), tuple(count))


def coarse_lattice(shape3, L):
    S = 1 << (L - 1)
    start, step, count = [0, 0, 0], [1, 1, 1], [1, 1, 1]
    for a in active_axes(shape3):
        step[a], count[a] = S, count_from(shape3[a], 0, S)
    return Lattice(tuple(start), tuple(step), tuple(count))


def sub_lattice(lat, u, v, su, tu, sv, tv):
    """Restrict ``lat`` to compact indices ku = su + tu*i, kv = sv + tv*j."""
    start, step, count = list(lat.start), list(lat.step), list(lat.count)
    for ax, s0, t in ((u, su, tu), (v, sv, tv)):
        start[ax] = lat.start[ax] + lat.step[ax] * s0
        step[ax] = lat.step[ax] * t
        count[ax] = count_from(lat.count[ax], s0, t)
    return Lattice(tuple(start), tuple(step), tuple(count))


# Coefficient decomposition sub-levels (Sec. V-B, Alg. 1): a 3-level 2-D
# per-level linear hierarchy on each slice.  In compact in-slice indices (u, v):
#   S1 = 4-grid (kept raw); S2 = 2-grid minus 4-grid; S3 = the rest.
# S2 and S3 each consist of two "regions" of the 2-D per-level scheme
# (odd along u first, then odd along v), concatenated in that order.
DECOMP_SUBLEVELS = (
    ((0, 4, 0, 4),),
    ((2, 4, 0, 4), (0, 2, 2, 4)),
    ((1, 2, 0, 2), (0, 1, 1, 2)),
)


def decomp_axes(decomp_axis):
    """In-slice axes (u, v) for slices normal to ``decomp_axis``."""
    return tuple(a for a in range(3) if a != decomp_axis)


@dataclass
class Stream:
    level: int
    region: int            # 0 for the coarse level or a whole per-level level
    sub: int               # 0 = no decomposition, 1..3 = S1..S3
    lattices: List[Lattice]
    is_int: bool           # fixed-point (levels >= 1) or field dtype (level 0)

    @property
    def n_real(self):
        return sum(l.n_real for l in self.lattices)

    @property
    def n_pad(self):
        return sum(l.n_pad for l in self.lattices)

    @property
    def words(self):
        return self.n_pad // WORD


@dataclass
class Geometry:
    shape3: Tuple[int, int, int]
    L: int
    interp: str            # "level" | "region"
    order: Tuple[int, ...]  # pass order over active axes
    decomp_axis: int       # -1 = none
    streams: List[Stream] = field(default_factory=list)

    @property
    def d(self):
        return len(self.order)


def build_geometry(shape3, L, interp, order, decomp_axis):
    """Streams in canonical order: levels L-1 .. 0; within a level, regions
    1..d; within a decomposed region, S1, S2, S3."""
    shape3 = tuple(int(x) for x in shape3)
    act = active_axes(shape3)
    assert sorted(order) == list(act), (order, act)
    if interp == "level":
        assert tuple(order) == act, "per-level interpolation uses the natural order"
    if decomp_axis >= 0:
        assert len(act) == 3 and decomp_axis in act
    g = Geometry(shape3, L, interp, tuple(order), decomp_axis)
    g.streams.append(Stream(L - 1, 0, 0, [coarse_lattice(shape3, L)], L - 1 >= 1))
    for level in range(L - 2, -1, -1):
        regions = [region_lattice(shape3, level, order, r) for r in range(1, len(order) + 1)]
        is_int = level >= 1
        if level == 0 and decomp_axis >= 0:
            u, v = decomp_axes(decomp_axis)
            for r, lat in enumerate(regions, start=1):
                for k, parts in enumerate(DECOMP_SUBLEVELS, start=1):
                    lats = [sub_lattice(lat, u, v, *p) for p in parts]
                    g.streams.append(Stream(0, r, k, lats, False))
        elif interp == "level":
            g.streams.append(Stream(level, 0, 0, regions, is_int))
        else:
            for r, lat in enumerate(regions, start=1):
                g.streams.append(Stream(level, r, 0, [lat], is_int))
    return g

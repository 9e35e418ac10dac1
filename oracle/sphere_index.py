"""CPU restatement of the spherical index (Brodu, "Spherical Indexing for
Neighborhood Queries").  TEST INFRASTRUCTURE ONLY: tests, the smoke check and
the benchmark's CPU-baseline leg may use it; no product path does.

It is written from the paper's text, step by step, in the paper's notation,
for small inputs (numpy, float64):

  * Sec. II.A, Fig. 2: the minimum-bound squared distance b^2 of every cell
    offset (cell units), the global offset array sorted by b^2 and the entry
    index by floor(d^2) ("end" array), with empty b^2 values aliasing to the
    entry below.
  * Sec. II.B: packed (ZYX bit concatenation) and unpacked (Y moved up by the
    packed width) cell locations; translation of an offset by add, mask and
    pack; n+1-bit offsets and one unique outside cell on non-cyclic axes.
  * Sec. III.A: 1-D shaving (frac(d) < zeta), the 64 specialized tables of
    Eq. 1 / Eq. 2, the run-time exact cell test above d - 1, and unconditional
    inclusion of cells lying wholly inside the sphere.
  * Sec. III.C: the parallelepiped (bin-lattice cube clipped to the region).

Two readings are taken where the paper is silent or unsafe:
  * Unconditional inclusion uses the exact farthest-corner distance of the
    target cell; the printed rule "b < d - sqrt(3)" can include a cell whose
    far corner lies outside the sphere (offset (10,0,0), b = 9, d = 10.8).
  * The center cell (offset 0) is never pre-rejected by a specialized table:
    Eq. 2 needs at least one direction with an offset.
The final per-object test is the canonical FP64 predicate (same definition
as brute.c, written again here).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# ---------------------------------------------------------------------------
# Sec. II.A -- minimum-bound squared distances and the sorted offset table
# ---------------------------------------------------------------------------


def min_bound_sq(offsets: np.ndarray) -> np.ndarray:
    """b^2 of each integer cell offset (Fig. 2): per axis the gap between the
    center cell and the target cell is max(|o| - 1, 0) cells; the points of
    the 3x3(x3) block around the center may touch, so their bound is 0."""
    gap = np.maximum(np.abs(offsets) - 1, 0)
    return (gap * gap).sum(axis=-1)


def fig2_grid(half: int = 4) -> np.ndarray:
    """The 2-D table of Fig. 2 for offsets -half..half on both axes."""
    o = np.arange(-half, half + 1)
    oy, ox = np.meshgrid(o, o, indexing="ij")
    return min_bound_sq(np.stack([ox, oy], axis=-1))


def axis_offset_range(w: int, cyclic: bool, reach: int) -> np.ndarray:
    """Offsets kept on one axis.  Non-cyclic: |o| <= min(reach, G - 1) (further
    offsets always leave the region).  Cyclic: |o| <= reach and the caller
    guarantees 2*reach + 1 <= G, so every cell of the ring appears once
    (Sec. III.C: no duplicates)."""
    g = 1 << w
    lim = min(reach, g - 1)
    return np.arange(-lim, lim + 1)


@dataclass
class OffsetTable:
    offsets: np.ndarray   # (E, 3) int64 offsets (x, y, z), sorted by b^2
    b2: np.ndarray        # (E,) int64
    end: np.ndarray       # end[n] = number of entries with b^2 <= n, n = 0..n_max
    n_max: int


def build_offset_table(n_max: int, log2_cells, cyclic_mask: int) -> OffsetTable:
    """Global offset array sorted by b^2 from center to edge, and the index by
    floor(d^2): entries for b^2 <= n are exactly offsets[:end[n]] (Sec. II.A)."""
    reach = math.isqrt(n_max) + 1          # b_i <= sqrt(n_max)  =>  |o_i| <= isqrt + 1
    axes = []
    for a in range(3):
        cyc = bool((cyclic_mask >> a) & 1)
        if cyc and 2 * reach + 1 > (1 << log2_cells[a]):
            raise ValueError("radius covers the whole cyclic axis (whole-world regime)")
        axes.append(axis_offset_range(log2_cells[a], cyc, reach))
    oz, oy, ox = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    off = np.stack([ox.ravel(), oy.ravel(), oz.ravel()], axis=1).astype(np.int64)
    b2 = min_bound_sq(off)
    keep = b2 <= n_max
    off, b2 = off[keep], b2[keep]
    order = np.lexsort((off[:, 0], off[:, 1], off[:, 2], b2))
    off, b2 = off[order], b2[order]
    end = np.searchsorted(b2, np.arange(n_max + 1), side="right")
    return OffsetTable(off, b2, end, n_max)


def shell_counts(table: OffsetTable) -> dict:
    """Number of offsets at each b^2 value (Fig. 2 text: 27, 54, 36, 8, 54, ...)."""
    vals, cnt = np.unique(table.b2, return_counts=True)
    return {int(v): int(c) for v, c in zip(vals, cnt)}


# ---------------------------------------------------------------------------
# Sec. III.A -- the 64 specialized tables (Eq. 1 / Eq. 2)
# ---------------------------------------------------------------------------

def direction_bits(off: np.ndarray) -> np.ndarray:
    """Bit 2*axis + (1 if the offset is negative on that axis) for every axis on
    which the offset is non-zero."""
    bits = np.zeros(off.shape[0], dtype=np.int64)
    for a in range(3):
        bits |= np.where(off[:, a] > 0, 1 << (2 * a), 0)
        bits |= np.where(off[:, a] < 0, 1 << (2 * a + 1), 0)
    return bits


@dataclass
class SpecializedTables:
    """For each floor(d) value fl and each 6-bit mask: the entries of the shell
    fl^2 <= b^2 < (fl+1)^2 that Eq. 2 does NOT pre-reject, in table order."""
    lists: dict           # (fl, mask) -> np.ndarray of indices into OffsetTable


def build_specialized_tables(table: OffsetTable) -> SpecializedTables:
    dirs = direction_bits(table.offsets)
    nonzero = np.any(table.offsets != 0, axis=1)
    lists = {}
    fl_max = math.isqrt(table.n_max)
    for fl in range(fl_max + 1):
        lo, hi = fl * fl, (fl + 1) * (fl + 1)
        idx = np.nonzero((table.b2 >= lo) & (table.b2 < hi) & (table.b2 <= table.n_max))[0]
        for mask in range(64):
            # Eq. 2: with b >= floor(d) and f < zeta_i on every direction the
            # offset points to, t > d, so the cell is rejected beforehand.
            rejected = nonzero[idx] & ((dirs[idx] & ~mask) == 0)
            lists[(fl, mask)] = idx[~rejected]
    return SpecializedTables(lists)


# ---------------------------------------------------------------------------
# Sec. II.B -- packed / unpacked cell locations
# ---------------------------------------------------------------------------

@dataclass
class Lattice:
    log2_cells: tuple     # (wx, wy, wz)
    cyclic_mask: int

    @property
    def W(self) -> int:
        return sum(self.log2_cells)

    @property
    def outside(self) -> int:
        """The unique extra cell holding every object outside the region."""
        return 1 << self.W


def pack(cx, cy, cz, lat: Lattice):
    """Packed location: bits z | y | x (ZYX order), also the memory index."""
    wx, wy, _ = lat.log2_cells
    return (cz << (wx + wy)) | (cy << wx) | cx


def unpack(packed, lat: Lattice):
    """Unpacked location: the Y bits moved left by the packed width W, leaving
    zero gaps that absorb carries when an offset is added."""
    wx, wy, _ = lat.log2_cells
    ymask = ((1 << wy) - 1) << wx
    return (packed & ~ymask) | ((packed & ymask) << lat.W)


def field_positions(lat: Lattice):
    wx, wy, _ = lat.log2_cells
    return (0, lat.W + wx, wx + wy)       # bit position of x, y, z in unpacked form


def offset_unpacked(off, lat: Lattice):
    """Offset (ox, oy, oz) in unpacked form: two's complement on w bits for a
    cyclic axis and on w + 1 bits for a non-cyclic axis."""
    pos = field_positions(lat)
    out = 0
    for a in range(3):
        w = lat.log2_cells[a] + (0 if (lat.cyclic_mask >> a) & 1 else 1)
        out |= (int(off[a]) & ((1 << w) - 1)) << pos[a]
    return out


def valid_mask(lat: Lattice):
    pos = field_positions(lat)
    m = 0
    for a in range(3):
        m |= ((1 << lat.log2_cells[a]) - 1) << pos[a]
    return m


def guard_mask(lat: Lattice):
    """Bit w of every non-cyclic field: set after the add iff that coordinate
    left [0, G)."""
    pos = field_positions(lat)
    m = 0
    for a in range(3):
        if not (lat.cyclic_mask >> a) & 1:
            m |= 1 << (pos[a] + lat.log2_cells[a])
    return m


def translate(center_unpacked, off_unpacked, lat: Lattice):
    """Add, mask out the two's-complement overflow, pack (Sec. II.B).  On a
    non-cyclic axis a set guard bit sends the cell to the outside cell."""
    s = center_unpacked + off_unpacked
    outside = (s & guard_mask(lat)) != 0
    s = s & valid_mask(lat)
    W = lat.W
    packed = (s >> W) | (s & ((1 << W) - 1))
    return np.where(outside, lat.outside, packed) if isinstance(s, np.ndarray) else (
        lat.outside if outside else packed)


# ---------------------------------------------------------------------------
# Canonical predicate (same definition as brute.c, restated)
# ---------------------------------------------------------------------------

def canon_d2(qi: np.ndarray, pj: np.ndarray, L, cyclic_mask: int) -> np.ndarray:
    """FP64 squared distance, per-axis shorter way round on cyclic axes."""
    acc = None
    for a in range(3):
        g = np.abs(pj[..., a].astype(np.float64) - qi[..., a].astype(np.float64))
        if (cyclic_mask >> a) & 1:
            g = np.minimum(g, float(L[a]) - g)
        sq = g * g
        acc = sq if acc is None else acc + sq
    return acc


# ---------------------------------------------------------------------------
# Binning and the query walk
# ---------------------------------------------------------------------------

@dataclass
class CpuGrid:
    lat: Lattice
    origin: np.ndarray    # (3,) float64
    s: float              # cell side
    L: np.ndarray         # (3,) float64 box side per axis
    pos: np.ndarray       # (n, 4) float32, input order
    key: np.ndarray       # (n,) cell of each object (packed, or outside)
    order: np.ndarray     # object indices sorted by cell (stable)
    start: np.ndarray     # (cells + 1 + 1,) start[c] .. start[c+1] in `order`


def cell_coords(pos: np.ndarray, origin, s: float, lat: Lattice):
    """Integer cell coordinates (float64 floor) and in-region flags."""
    rel = pos[:, :3].astype(np.float64) - np.asarray(origin, dtype=np.float64)
    u = rel / s
    c = np.floor(u).astype(np.int64)
    inside = np.ones(pos.shape[0], dtype=bool)
    for a in range(3):
        g = 1 << lat.log2_cells[a]
        if (lat.cyclic_mask >> a) & 1:
            if np.any((c[:, a] < 0) | (c[:, a] >= g)):
                raise ValueError("cyclic-axis coordinate outside the box")
        else:
            inside &= (c[:, a] >= 0) & (c[:, a] < g)
    return c, u - c, inside


def build_cpu_grid(pos, origin, s, log2_cells, cyclic_mask) -> CpuGrid:
    lat = Lattice(tuple(log2_cells), cyclic_mask)
    c, _, inside = cell_coords(pos, origin, s, lat)
    key = np.where(inside, pack(c[:, 0], c[:, 1], c[:, 2], lat), lat.outside)
    order = np.argsort(key, kind="stable")
    ncell = lat.outside + 1
    counts = np.bincount(key, minlength=ncell)
    start = np.zeros(ncell + 1, dtype=np.int64)
    np.cumsum(counts, out=start[1:])
    L = np.array([float(np.float32(s) * np.float32(1 << w)) for w in log2_cells])
    return CpuGrid(lat, np.asarray(origin, np.float64), float(s), L, pos, key, order, start)


MARGIN = 1e-9   # cell units; float64 rounding of the cell arithmetic is ~1e-14


def sphere_cells(grid: CpuGrid, center, d: float, table: OffsetTable,
                 spec: SpecializedTables, runtime_test_from: float | None = None):
    """Cells the spherical index visits for one in-region query center.

    Returns (cells, inside_flags) where inside_flags marks cells whose every
    point is within d (unconditional inclusion).  Center-to-edge order."""
    lat = grid.lat
    u = (np.asarray(center[:3], np.float64) - grid.origin) / grid.s
    c = np.floor(u).astype(np.int64)
    phi = u - c
    n = int(math.floor(d * d))
    if n > table.n_max:
        raise ValueError("radius beyond the table")
    fl = math.isqrt(n)
    f = d - fl
    zeta_pos, zeta_neg = 1.0 - phi, phi
    mask = 0
    for a in range(3):
        if f < zeta_pos[a] - MARGIN:
            mask |= 1 << (2 * a)
        if f < zeta_neg[a] - MARGIN:
            mask |= 1 << (2 * a + 1)
    # main table below floor(d), then the specialized table of the shell
    main = np.arange(table.end[fl * fl - 1] if fl > 0 else 0)
    tail = spec.lists[(fl, mask)]
    tail = tail[table.b2[tail] <= n]
    idx = np.concatenate([main, tail])
    off = table.offsets[idx]
    b2 = table.b2[idx]
    # run-time exact test (Sec. III.A) for cells with b > d - 1 by default
    thr = (d - 1.0) if runtime_test_from is None else runtime_test_from
    b = np.sqrt(b2.astype(np.float64))
    zeta = np.where(off > 0, zeta_pos, np.where(off < 0, zeta_neg, 0.0))
    gap = np.where(off != 0, np.maximum(np.abs(off) - 1, 0) + zeta, 0.0)
    t2 = (gap * gap).sum(axis=1)
    keep = ~((b > thr) & (t2 > (d + MARGIN) ** 2))
    off, b2 = off[keep], b2[keep]
    # farthest point of the target cell, for unconditional inclusion
    far = np.maximum(np.abs(off - phi), np.abs(off + 1 - phi))
    inside = (far * far).sum(axis=1) <= (d - MARGIN) ** 2
    cu = unpack(int(pack(c[0], c[1], c[2], lat)), lat)
    cells = np.array([translate(cu, offset_unpacked(o, lat), lat) for o in off], dtype=np.int64)
    inside = inside & (cells != lat.outside)
    return cells, inside


def _in_region(center, grid: CpuGrid) -> bool:
    u = (np.asarray(center[:3], np.float64) - grid.origin) / grid.s
    for a in range(3):
        if not (grid.lat.cyclic_mask >> a) & 1:
            if not (0 <= u[a] < (1 << grid.lat.log2_cells[a])):
                return False
    return True


def parallelepiped_cells(grid: CpuGrid, center, d: float):
    """Bin-lattice cells: the bounding cube of the sphere, clipped to the region
    on non-cyclic axes (Sec. III.C), wrapped on cyclic axes; plus the outside
    cell when the cube leaves the region."""
    lat = grid.lat
    u = (np.asarray(center[:3], np.float64) - grid.origin) / grid.s
    ranges, leaves = [], False
    for a in range(3):
        g = 1 << lat.log2_cells[a]
        lo, hi = int(math.floor(u[a] - d - MARGIN)), int(math.floor(u[a] + d + MARGIN))
        if (lat.cyclic_mask >> a) & 1:
            ranges.append(np.arange(lo, hi + 1) % g)
        else:
            if lo < 0 or hi >= g:
                leaves = True
            ranges.append(np.arange(max(lo, 0), min(hi, g - 1) + 1))
    cz, cy, cx = np.meshgrid(ranges[2], ranges[1], ranges[0], indexing="ij")
    cells = pack(cx.ravel(), cy.ravel(), cz.ravel(), lat)
    if leaves:
        cells = np.concatenate([cells, [lat.outside]])
    return np.unique(cells)


def query_radius(grid: CpuGrid, centers: np.ndarray, r: float, self_idx=None,
                 method: str = "sphere", n_max: int | None = None):
    """Radius query through the spherical index (or the parallelepiped scan).
    Returns (offsets, ids) CSR with ids ascending, plus visited-cell counts."""
    d = r / grid.s
    n_tab = int(math.floor(d * d)) if n_max is None else n_max
    table = build_offset_table(n_tab, grid.lat.log2_cells, grid.lat.cyclic_mask)
    spec = build_specialized_tables(table)
    r2 = float(r) * float(r)
    lists, visited = [], []
    for k in range(centers.shape[0]):
        ctr = centers[k]
        if method == "sphere" and _in_region(ctr, grid):
            cells, full = sphere_cells(grid, ctr, d, table, spec)
            # the outside cell is visited once however many offsets reach it
            uniq, first = np.unique(cells, return_index=True)
            cells, full = uniq, full[first]
        else:
            cells = parallelepiped_cells(grid, ctr, d)
            full = np.zeros(cells.shape[0], dtype=bool)
        visited.append(cells.shape[0])
        found = []
        for cell, inc in zip(cells, full):
            members = grid.order[grid.start[cell]:grid.start[cell + 1]]
            if members.size == 0:
                continue
            if inc:
                found.append(members)
            else:
                dd = canon_d2(ctr[None, :], grid.pos[members], grid.L, grid.lat.cyclic_mask)
                found.append(members[dd <= r2])
        ids = np.sort(np.concatenate(found)) if found else np.zeros(0, np.int64)
        if self_idx is not None and self_idx[k] >= 0:
            ids = ids[ids != self_idx[k]]
        lists.append(ids)
    offsets = np.zeros(len(lists) + 1, dtype=np.int64)
    np.cumsum([x.size for x in lists], out=offsets[1:])
    ids = np.concatenate(lists).astype(np.int32) if lists else np.zeros(0, np.int32)
    return offsets, ids, np.array(visited)


def exact_cells_within(center_frac: np.ndarray, d: float, reach: int) -> int:
    """Number of cells whose exact distance from a point at sub-cell position
    center_frac is <= d (the ideal per-query culling), by enumeration."""
    o = np.arange(-reach, reach + 1)
    oz, oy, ox = np.meshgrid(o, o, o, indexing="ij")
    off = np.stack([ox.ravel(), oy.ravel(), oz.ravel()], axis=1)
    zeta = np.where(off > 0, 1.0 - center_frac, np.where(off < 0, center_frac, 0.0))
    gap = np.where(off != 0, np.maximum(np.abs(off) - 1, 0) + zeta, 0.0)
    return int(((gap * gap).sum(axis=1) <= d * d).sum())

"""Pins of the oracle's restatement of the spherical index against values the
paper prints (Fig. 2, Sec. II.A; the Sec. II.B worked example) and against
geometry (pi/6 limit, Steiner volume, Eq. 2 validity)."""
import math

import numpy as np
import pytest

from oracle import sphere_index as si


def test_fig2_min_bound_grid(golden):
    want = np.array([[int(v) for v in row] for row in golden("fig2_min_bound_2d.txt")])
    assert np.array_equal(si.fig2_grid(4), want)


def test_fig2_example_cells():
    # Fig. 2 caption: gray cells 3^2 + 2^2 = 13 and 2^2 + 1^2 = 5.
    assert si.min_bound_sq(np.array([4, 3])) == 13
    assert si.min_bound_sq(np.array([3, 2])) == 5


def test_3d_shell_counts_and_missing_entry(golden):
    t = si.build_offset_table(9, (8, 8, 8), 0)
    counts = si.shell_counts(t)
    for b2, c in golden("shell_counts_3d.txt"):
        assert counts.get(int(b2), 0) == int(c)
    # b^2 = 7 aliases to the entry below (Sec. II.A)
    assert t.end[7] == t.end[6]
    # end[] is the prefix count by construction: entries below or equal to n
    for n in range(10):
        assert t.end[n] == int((t.b2 <= n).sum())
    assert np.all(np.diff(t.b2) >= 0)


def test_swar_worked_example(golden):
    g = {row[0]: row[1:] for row in golden("swar_worked_example.txt")}
    wx, wy, wz = (int(v) for v in g["lattice_log2"])
    lat = si.Lattice((wx, wy, wz), 7)
    cx, cy, cz = (int(v) for v in g["cell"])
    bits = lambda key: int("".join(g[key]), 2)
    packed = si.pack(cx, cy, cz, lat)
    assert packed == bits("packed")
    unp = si.unpack(packed, lat)
    assert unp == bits("unpacked")
    off = si.offset_unpacked([int(v) for v in g["offset"]], lat)
    assert off == bits("offset_unpacked")
    assert unp + off == bits("sum")
    assert si.valid_mask(lat) == bits("mask")
    assert (unp + off) & si.valid_mask(lat) == bits("masked")
    res = si.translate(unp, off, lat)
    assert res == bits("result_packed")
    assert (res & 31, (res >> 5) & 15, res >> 9) == tuple(int(v) for v in g["result_cell"])


@pytest.mark.parametrize("mask", [0, 1, 2, 4, 3, 5, 6, 7])
def test_swar_translate_matches_axis_arithmetic(mask):
    rng = np.random.default_rng(mask)
    lat = si.Lattice((5, 3, 4), mask)
    G = [1 << w for w in lat.log2_cells]
    for _ in range(400):
        c = [int(rng.integers(0, g)) for g in G]
        o = []
        for a, g in enumerate(G):
            lim = (g - 1) // 2 if (mask >> a) & 1 else g - 1
            o.append(int(rng.integers(-lim, lim + 1)))
        got = si.translate(si.unpack(si.pack(*c, lat), lat), si.offset_unpacked(o, lat), lat)
        t = [c[a] + o[a] for a in range(3)]
        if any(not (mask >> a) & 1 and not (0 <= t[a] < G[a]) for a in range(3)):
            assert got == lat.outside
        else:
            t = [t[a] % G[a] for a in range(3)]
            assert got == si.pack(*t, lat)


def test_sphere_over_cube_ratio_tends_to_pi_over_6():
    # Sec. I: cells intersecting the sphere / cells of the bounding cube -> ~52%.
    ratios = []
    for d in (8, 16, 32):
        t = si.build_offset_table(d * d, (8, 8, 8), 0)
        cube = (2 * (d + 1) + 1) ** 3
        ratios.append(t.end[d * d] / cube)
    assert abs(ratios[-1] - math.pi / 6) < 0.01
    assert ratios[0] < ratios[1] < ratios[2] < math.pi / 6


def test_exact_culling_matches_steiner_volume():
    # Mean number of unit cells within distance d of a uniform random point is
    # the volume of the Minkowski sum of a unit cube and a ball of radius d:
    # 1 + 6 d + 3 pi d^2 + 4/3 pi d^3.
    rng = np.random.default_rng(5)
    for d in (0.5, 1.5, 2.5):
        vals = [si.exact_cells_within(rng.random(3), d, int(d) + 2) for _ in range(4000)]
        steiner = 1 + 6 * d + 3 * math.pi * d * d + 4 / 3 * math.pi * d ** 3
        se = np.std(vals) / math.sqrt(len(vals))
        assert abs(np.mean(vals) - steiner) < 4 * se + 1e-9


def test_specialized_tables_only_reject_cells_beyond_d():
    # Eq. 2: a pre-rejected cell of the shell floor(d) has true distance t > d.
    rng = np.random.default_rng(11)
    t = si.build_offset_table(16, (8, 8, 8), 0)
    spec = si.build_specialized_tables(t)
    for _ in range(3000):
        d = rng.uniform(0.05, 4.0)
        phi = rng.random(3)
        n = int(math.floor(d * d))
        fl = math.isqrt(n)
        f = d - fl
        mask = 0
        for a in range(3):
            mask |= (f < 1 - phi[a]) << (2 * a)
            mask |= (f < phi[a]) << (2 * a + 1)
        shell = np.nonzero((t.b2 >= fl * fl) & (t.b2 <= n))[0]
        kept = set(spec.lists[(fl, mask)].tolist())
        for e in shell:
            if e in kept:
                continue
            o = t.offsets[e]
            zeta = np.where(o > 0, 1 - phi, np.where(o < 0, phi, 0.0))
            gap = np.where(o != 0, np.maximum(np.abs(o) - 1, 0) + zeta, 0.0)
            assert (gap * gap).sum() > d * d


def test_sphere_walk_is_conservative_and_tighter_than_cube():
    rng = np.random.default_rng(3)
    lat = (5, 5, 5)
    pos = np.zeros((1, 4), np.float32)
    g = si.build_cpu_grid(pos, (0, 0, 0), 1.0, lat, 7)
    for d in (0.4, 0.9, 1.5, 2.3, 3.7):
        t = si.build_offset_table(int(d * d), lat, 7)
        spec = si.build_specialized_tables(t)
        for _ in range(200):
            ctr = np.concatenate([rng.random(3) * 32, [0]]).astype(np.float32)
            cells, _ = si.sphere_cells(g, ctr, d, t, spec)
            cube = si.parallelepiped_cells(g, ctr, d)
            assert set(cells.tolist()) <= set(cube.tolist())
            # every cell within exact distance d is visited
            u = ctr[:3].astype(np.float64)
            c = np.floor(u).astype(int)
            phi = u - c
            R = int(d) + 2
            for ox in range(-R, R + 1):
                for oy in range(-R, R + 1):
                    for oz in range(-R, R + 1):
                        o = np.array([ox, oy, oz])
                        zeta = np.where(o > 0, 1 - phi, np.where(o < 0, phi, 0.0))
                        gap = np.where(o != 0, np.maximum(np.abs(o) - 1, 0) + zeta, 0.0)
                        if (gap * gap).sum() <= d * d:
                            tc = (c + o) % 32
                            assert si.pack(*tc, g.lat) in set(cells.tolist())

"""Pins of the FP64 brute-force oracle against an independent algorithm (the
paper's spherical index restated on the CPU), a library routine (scipy's
periodic k-d tree), closed forms and invariants."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from oracle import sphere_index as si
from paper_cs_0608108_b300 import synth

UNIT = (1.0, 1.0, 1.0)


def _lists(off, ids):
    return [ids[off[k]:off[k + 1]] for k in range(len(off) - 1)]


@pytest.mark.parametrize("mask", [0, 7, 3, 6])
def test_brute_matches_sphere_index_and_parallelepiped(mask):
    pos = synth.uniform_points(2500, 100 + mask)
    if not mask & 4:
        pos[:4, 2] = np.float32(1.03)    # outside the region on z
    if not mask & 1:
        pos[4:7, 0] = np.float32(-0.02)  # outside on x
    r = 0.085
    self_idx = np.arange(pos.shape[0])
    off_b, ids_b = oracle.radius(pos, pos, UNIT, mask, r, self_idx)
    g = si.build_cpu_grid(pos, (0, 0, 0), 1 / 16, (4, 4, 4), mask)
    off_s, ids_s, vis_s = si.query_radius(g, pos, r, self_idx, "sphere")
    off_c, ids_c, vis_c = si.query_radius(g, pos, r, self_idx, "cube")
    assert np.array_equal(off_b, off_s) and np.array_equal(ids_b, ids_s)
    assert np.array_equal(off_b, off_c) and np.array_equal(ids_b, ids_c)
    assert vis_s.mean() < vis_c.mean()


def _safe_radius(pos, box, periodic, r0):
    """A radius with no pair distance within 1e-9 relative of it, so that a
    library's own rounding cannot flip a boundary decision."""
    tree = cKDTree(pos[:, :3].astype(np.float64), boxsize=box if periodic else None)
    r = r0
    for _ in range(50):
        dd = tree.sparse_distance_matrix(tree, r * 1.000001, output_type="ndarray")["v"]
        if not np.any(np.abs(dd - r) < 1e-9 * r):
            return r
        r *= 1.0001
    raise AssertionError("no safe radius")


@pytest.mark.parametrize("periodic", [True, False])
def test_brute_matches_scipy_kdtree(periodic):
    pos = synth.uniform_points(4000, 7 if periodic else 8)
    mask = 7 if periodic else 0
    r = _safe_radius(pos, UNIT, periodic, 0.07)
    off, ids = oracle.radius(pos, pos, UNIT, mask, r, np.arange(4000))
    tree = cKDTree(pos[:, :3].astype(np.float64), boxsize=UNIT if periodic else None)
    for k, lst in enumerate(_lists(off, ids)):
        want = sorted(j for j in tree.query_ball_point(pos[k, :3].astype(np.float64), r) if j != k)
        assert lst.tolist() == want


def test_knn_matches_scipy_kdtree():
    pos = synth.uniform_points(3000, 21)
    k = 8
    ids, d2, cnt = oracle.knn(pos, pos, UNIT, 7, k, None, np.arange(3000))
    tree = cKDTree(pos[:, :3].astype(np.float64), boxsize=UNIT)
    dist, nbr = tree.query(pos[:, :3].astype(np.float64), k=k + 1)
    assert np.all(cnt == k)
    # drop self (distance 0 at column 0 unless duplicates exist)
    assert np.allclose(np.sqrt(d2), dist[:, 1:], rtol=1e-12, atol=1e-15)
    distinct = np.all(np.diff(dist[:, 1:], axis=1) > 1e-12, axis=1)
    assert distinct.mean() > 0.99
    assert np.array_equal(ids[distinct], nbr[distinct, 1:])


def test_knn_is_prefix_of_sorted_radius_list_with_id_ties():
    # coordinates on a coarse grid produce many exact distance ties
    rng = np.random.default_rng(4)
    pos = np.zeros((600, 4), np.float32)
    pos[:, :3] = rng.integers(0, 16, size=(600, 3)) / 16.0
    r = 0.2
    off, ids = oracle.radius(pos, pos, UNIT, 5, r, np.arange(600))
    kid, kd2, kc = oracle.knn(pos, pos, UNIT, 5, 6, r, np.arange(600))
    ties = 0
    for q, lst in enumerate(_lists(off, ids)):
        d2 = np.array([oracle.canon_d2(pos[q], pos[j], UNIT, 5) for j in lst])
        order = np.lexsort((lst, d2))
        want = lst[order][:6]
        assert kc[q] == min(6, len(lst))
        assert kid[q, :kc[q]].tolist() == want.tolist()
        assert np.all(kid[q, kc[q]:] == -1)
        ties += len(d2) - len(np.unique(d2))
    assert ties > 100


def test_unbounded_knn_counts_and_symmetry():
    pos = synth.uniform_points(500, 9)
    _, _, cnt = oracle.knn(pos, pos, UNIT, 0, 8, None, np.arange(500))
    assert np.all(cnt == 8)
    off, ids = oracle.radius(pos, pos, UNIT, 0, 2.0, np.arange(500))   # r > box diagonal
    assert np.all(np.diff(off) == 499)


def test_radius_relation_is_symmetric():
    pos = synth.uniform_points(3000, 31)
    for mask in (0, 7, 2):
        off, ids = oracle.radius(pos, pos, UNIT, mask, 0.08, np.arange(3000))
        pairs = set()
        for q, lst in enumerate(_lists(off, ids)):
            pairs.update((q, int(j)) for j in lst)
        assert all((j, q) in pairs for q, j in pairs)
        assert len(pairs) % 2 == 0


def test_translation_invariance_under_cyclic_wrap():
    # positions on a 2^-20 grid: shifts by multiples of 2^-20 and the wrap are
    # exact in FP32 and FP64, so distances (and sets) must not change
    rng = np.random.default_rng(12)
    n = 2000
    grid = rng.integers(0, 1 << 20, size=(n, 3))
    pos = np.zeros((n, 4), np.float32)
    pos[:, :3] = grid * 2.0 ** -20
    off0, ids0 = oracle.radius(pos, pos, UNIT, 7, 0.07, np.arange(n))
    for shift in ([12345, 0, 0], [0, 700001, 3], [524288, 524288, 999999]):
        moved = np.zeros_like(pos)
        moved[:, :3] = ((grid + np.array(shift)) % (1 << 20)) * 2.0 ** -20
        off1, ids1 = oracle.radius(moved, moved, UNIT, 7, 0.07, np.arange(n))
        assert np.array_equal(off0, off1) and np.array_equal(ids0, ids1)


def test_boundary_is_inclusive():
    # Sec. II.A: objects with x <= d are neighbors
    pos = np.array([[0.25, 0.5, 0.5, 0], [0.375, 0.5, 0.5, 0], [0.5, 0.5, 0.5, 0]], np.float32)
    off, ids = oracle.radius(pos, pos[:1], UNIT, 0, 0.125, [0])
    assert ids.tolist() == [1]
    off, ids = oracle.radius(pos, pos[:1], UNIT, 0, float(np.nextafter(0.125, 0)), [0])
    assert ids.tolist() == []
    # cyclic: 0.0625 and 0.9375 are 0.125 apart the short way round
    pos = np.array([[0.0625, 0.5, 0.5, 0], [0.9375, 0.5, 0.5, 0]], np.float32)
    assert oracle.radius(pos, pos[:1], UNIT, 1, 0.125, [0])[1].tolist() == [1]
    assert oracle.radius(pos, pos[:1], UNIT, 0, 0.125, [0])[1].tolist() == []


# ---------------------------------------------------------------------------
# smooth reduction: closed forms, finite differences, invariants
# ---------------------------------------------------------------------------

def test_reduce_two_and_three_point_closed_forms():
    r = 0.1
    pos = np.array([[0.5, 0.5, 0.5, 0], [0.55, 0.5, 0.5, 0]], np.float32)
    dlt = float(pos[1, 0]) - float(pos[0, 0])
    e, g = oracle.reduce(pos, [0, 1], UNIT, 0, r)
    w = (1 - dlt * dlt / (r * r)) ** 3
    assert math.isclose(e.sum(), 2 * w, rel_tol=1e-12)
    gx = -12 / (r * r) * (1 - dlt * dlt / (r * r)) ** 2 * (-dlt)
    assert math.isclose(g[0, 0], gx, rel_tol=1e-12) and math.isclose(g[1, 0], -gx, rel_tol=1e-12)
    assert g[0, 1] == 0 and g[0, 2] == 0
    # three collinear points, outer pair beyond r
    pos = np.array([[0.3, 0.5, 0.5, 0], [0.36, 0.5, 0.5, 0], [0.42, 0.5, 0.5, 0]], np.float32)
    e, g = oracle.reduce(pos, [0, 1, 2], UNIT, 0, r)
    a = float(pos[1, 0]) - float(pos[0, 0])
    b = float(pos[2, 0]) - float(pos[1, 0])
    want = 2 * (1 - a * a / r / r) ** 3 + 2 * (1 - b * b / r / r) ** 3
    assert math.isclose(e.sum(), want, rel_tol=1e-12)
    assert abs(g[:, 0].sum()) < 1e-9 * np.abs(g).max()


def test_reduce_two_points_across_the_wrap():
    r = 0.1
    pos = np.array([[0.02, 0.5, 0.5, 0], [0.97, 0.5, 0.5, 0]], np.float32)
    e, g = oracle.reduce(pos, [0, 1], UNIT, 1, r)
    dlt = 1.0 - (float(pos[1, 0]) - float(pos[0, 0]))
    assert math.isclose(e.sum(), 2 * (1 - dlt * dlt / (r * r)) ** 3, rel_tol=1e-12)
    # the short way round, point 0 sits 0.05 to the right of point 1
    assert g[0, 0] < 0 < g[1, 0]
    e0, _ = oracle.reduce(pos, [0, 1], UNIT, 0, r)
    assert e0.sum() == 0.0


def _energy(pos, mask, r):
    e, _ = oracle.reduce(pos, np.arange(pos.shape[0]), UNIT, mask, r)
    return e.sum()


@pytest.mark.parametrize("mask", [7, 0])
def test_reduce_gradient_matches_central_differences(mask):
    # positions on a 2^-24 grid, step h = 2^-16: x +- h stays exact in FP32
    pos = synth.uniform_points(400, 77 + mask)
    r = 0.12
    idx = np.arange(0, 400, 37)
    _, g = oracle.reduce(pos, idx, UNIT, mask, r)
    h = 2.0 ** -16
    for t, i in enumerate(idx):
        for a in range(3):
            p1, p0 = pos.copy(), pos.copy()
            p1[i, a] += np.float32(h)
            p0[i, a] -= np.float32(h)
            if mask and not (0 <= p1[i, a] < 1 and 0 <= p0[i, a] < 1):
                continue
            fd = (_energy(p1, mask, r) - _energy(p0, mask, r)) / (2 * h)
            assert abs(fd - g[t, a]) <= 1e-5 * max(1.0, abs(g[t, a]))


def test_reduce_invariants():
    pos = synth.uniform_points(1500, 5)
    e, g = oracle.reduce(pos, np.arange(1500), UNIT, 7, 0.1)
    assert np.all(e >= 0)
    assert np.abs(g.sum(axis=0)).max() < 1e-9 * np.abs(g).max()
    # every pair within r contributes: e_i > 0 exactly when i has a neighbor
    off, _ = oracle.radius(pos, pos, UNIT, 7, float(np.nextafter(0.1, 0)), np.arange(1500))
    assert np.array_equal(e > 0, np.diff(off) > 0)


@pytest.mark.parametrize("periodic", [True, False])
def test_queries_from_arbitrary_centers_match_scipy_kdtree(periodic):
    """Caller-given centers (nothing excluded; a center on a point finds it):
    radius lists and K nearest against an independent k-d tree."""
    pos = synth.uniform_points(3000, 31 if periodic else 32)
    cen = synth.uniform_points(1500, 33)
    cen[:10] = pos[:10]                          # centers on top of points
    mask = 7 if periodic else 0
    tp = cKDTree(pos[:, :3].astype(np.float64), boxsize=UNIT if periodic else None)
    tc = cKDTree(cen[:, :3].astype(np.float64), boxsize=UNIT if periodic else None)
    r = 0.06
    for _ in range(50):                          # a radius no center-point distance sits on
        dd = tc.sparse_distance_matrix(tp, r * 1.000001, output_type="ndarray")["v"]
        if not np.any(np.abs(dd - r) < 1e-9 * r):
            break
        r *= 1.0001
    off, ids = oracle.radius(pos, cen, UNIT, mask, r, None)
    for k, lst in enumerate(_lists(off, ids)):
        want = sorted(tp.query_ball_point(cen[k, :3].astype(np.float64), r))
        assert lst.tolist() == want
    assert all(k in _lists(off, ids)[k].tolist() for k in range(10))
    kk = 6
    kid, kd2, kcnt = oracle.knn(pos, cen, UNIT, mask, kk, None, None)
    dist, nbr = tp.query(cen[:, :3].astype(np.float64), k=kk)
    assert np.all(kcnt == kk)
    assert np.allclose(np.sqrt(kd2), dist, rtol=1e-12, atol=1e-15)
    distinct = np.all(np.diff(dist, axis=1) > 1e-12, axis=1)
    assert np.array_equal(kid[distinct], nbr[distinct])
    assert np.all(kid[:10, 0] == np.arange(10))   # distance 0 first


@pytest.mark.parametrize("mask", [7, 0, 5, 2])
def test_reduce_through_the_bin_lattice_equals_brute_force(mask):
    # the bin-lattice reduction (cells at least r wide) finds the same pairs
    # as the O(n^2) scan: per-object energies and gradients equal up to the
    # order of each FP64 sum; outside points on the non-cyclic axes, and a
    # radius for which a cyclic axis holds fewer than 3 cells (brute-force
    # fallback)
    pos = synth.uniform_points(3000, 70 + mask)
    for a in range(3):
        if not (mask >> a) & 1:
            pos[a * 7:(a + 1) * 7, a] = np.float32(1.3 if a % 2 else -0.4)
    box = (1.0, 1.0, 1.0)
    for r in (0.06, 0.35):
        e1, g1 = oracle.reduce(pos, np.arange(3000), box, mask, r)
        e2, g2 = oracle.reduce_all(pos, box, mask, r)
        assert np.allclose(e1, e2, rtol=1e-12, atol=1e-15)
        assert np.allclose(g1, g2, rtol=1e-12, atol=1e-12 * np.abs(g1).max())
        assert e1.sum() > 0

"""Parity of the CUDA binning and all-agents radius query with the FP64 oracle:
neighbor sets and counts bit-exact (ids ascending per query)."""
import math

import numpy as np
import pytest
import torch

from paper_cs_0608108_b300 import Grid, synth, _native

from gpu_helpers import (assert_csr_equal, assert_sampled_equal, gpu_grid, gpu_radius,
                         oracle_radius, to_dev)

pytestmark = pytest.mark.gpu


def test_binning_is_a_cell_ordered_permutation():
    sc = synth.uniform_points(50_000, 3)
    scene = synth.Scene(sc, (0, 0, 0), 1 / 32, (5, 5, 5), 0, 0.05)
    scene.pos[:7, 2] = np.float32(1.5)          # outside on z
    g = gpu_grid(scene)
    start, spos, perm = (t.cpu().numpy() for t in g.cell_arrays())
    g.sync()
    n = scene.n
    assert start[0] == 0 and start[-1] == n and np.all(np.diff(start) >= 0)
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert np.array_equal(spos, scene.pos[perm])
    # every point sits in (or within float rounding of) the cell it was binned in
    cells = np.repeat(np.arange(start.size - 1), np.diff(start))
    outside = 1 << 15
    u = scene.pos[perm, :3].astype(np.float64) * 32
    inside = cells != outside
    c = np.stack([cells & 31, (cells >> 5) & 31, cells >> 10], axis=1)[inside]
    assert np.all(u[inside] >= c - 1e-5) and np.all(u[inside] < c + 1 + 1e-5)
    assert set(perm[~inside].tolist()) == set(range(7))


WALKS = [("sphere", "classes"), ("sphere", "paper"), ("cube", "classes")]


def test_tiny_config_sphere_and_cube_bit_exact():
    # N=20k uniform, 32^3 non-cyclic, r = 0.03 (0.96 cells)
    scene = synth.tiny_scene()
    off_o, ids_o = oracle_radius(scene)
    for method, walk in WALKS:
        off_g, ids_g = gpu_radius(scene, method=method, walk=walk)
        assert_csr_equal(off_g, ids_g, off_o, ids_o)


@pytest.mark.parametrize("mask", [0, 1, 2, 4, 3, 5, 6, 7])
@pytest.mark.parametrize("r_cells", [0.45, 1.5, 2.7])
def test_every_cyclic_mask_and_radius(mask, r_cells):
    pos = synth.uniform_points(12_000, 1000 + mask)
    # points outside the region on every non-cyclic axis
    for a in range(3):
        if not (mask >> a) & 1:
            pos[a * 5:(a + 1) * 5, a] = np.float32(1.07 if a % 2 else -0.03)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), mask, r_cells / 16)
    off_o, ids_o = oracle_radius(scene)
    for method, walk in WALKS:
        off_g, ids_g = gpu_radius(scene, method=method, walk=walk)
        assert_csr_equal(off_g, ids_g, off_o, ids_o)


def test_non_power_of_two_box_and_offset_origin():
    # cell side 0.37 (box 5.92), origin (-2, 1, 3): float32 binning is inexact
    n = 15_000
    base = synth.uniform_points(n, 77, box=(5.92, 5.92, 5.92), origin=(-2.0, 1.0, 3.0))
    for mask in (7, 0, 5):
        scene = synth.Scene(base.copy(), (-2.0, 1.0, 3.0), 0.37, (4, 4, 4), mask, 0.37 * 1.7)
        off_o, ids_o = oracle_radius(scene)
        for method, walk in WALKS:
            off_g, ids_g = gpu_radius(scene, method=method, walk=walk)
            assert_csr_equal(off_g, ids_g, off_o, ids_o)


def test_guard_band_pairs_at_the_radius():
    # pairs at |d^2 - r^2| ~ 1e-7 r^2 (inside the FP32 band) must follow the FP64 predicate
    rng = np.random.default_rng(9)
    r = np.float32(1.5 / 64)
    m = 3000
    a = rng.random((m, 3)).astype(np.float32) * np.float32(0.9) + np.float32(0.05)
    direc = rng.normal(size=(m, 3))
    direc /= np.linalg.norm(direc, axis=1, keepdims=True)
    scale = 1.0 + rng.choice([-1, 1], size=m) * rng.uniform(1e-8, 3e-7, size=m)
    b = (a.astype(np.float64) + direc * float(r) * scale[:, None]).astype(np.float32)
    pos = np.zeros((2 * m, 4), np.float32)
    pos[0::2, :3] = a
    pos[1::2, :3] = np.mod(b, 1.0).astype(np.float32)
    pos[:, :3] = np.where(pos[:, :3] >= 1.0, np.float32(0), pos[:, :3])
    for mask in (7, 0):
        scene = synth.Scene(pos, (0, 0, 0), 1 / 64, (6, 6, 6), mask, float(r))
        off_o, ids_o = oracle_radius(scene)
        for method, walk in WALKS:
            off_g, ids_g = gpu_radius(scene, method=method, walk=walk)
            assert_csr_equal(off_g, ids_g, off_o, ids_o)
        assert 0 < off_o[-1] < 2 * m


def test_wrapped_pairs_near_the_radius():
    # pairs straddling the cyclic boundary at distance ~r (the wider wrapped band)
    rng = np.random.default_rng(5)
    m = 4000
    r = 2.0 / 128
    x = rng.uniform(0, 1, size=(m, 3))
    x[:, 0] = rng.uniform(0, r, size=m)
    y = x.copy()
    y[:, 0] = x[:, 0] - r * (1 + rng.uniform(-3e-6, 3e-6, size=m))
    y[:, 0] = np.mod(y[:, 0], 1.0)
    pos = np.zeros((2 * m, 4), np.float32)
    pos[0::2, :3] = x
    pos[1::2, :3] = y
    pos[:, :3] = np.where(pos[:, :3] >= 1.0, np.float32(0), pos[:, :3])
    scene = synth.Scene(pos, (0, 0, 0), 1 / 128, (7, 7, 7), 7, r)
    off_o, ids_o = oracle_radius(scene)
    for method, walk in WALKS:
        off_g, ids_g = gpu_radius(scene, method=method, walk=walk)
        assert_csr_equal(off_g, ids_g, off_o, ids_o)


@pytest.mark.parametrize("n", [0, 1, 2, 31, 33, 257])
def test_ragged_and_tiny_point_counts(n):
    pos = synth.uniform_points(max(n, 1), 11 + n)[:n]
    scene = synth.Scene(pos, (0, 0, 0), 1 / 8, (3, 3, 3), 7, 0.3)
    g = Grid(scene.origin, scene.cell_size, scene.log2_cells, 7, scene.r, max(n, 1))
    g.build(to_dev(pos))
    off, ids = g.query_radius(scene.r)
    g.sync()
    off_o, ids_o = oracle_radius(scene)
    assert_csr_equal(off.cpu().numpy(), ids.cpu().numpy(), off_o, ids_o)


def test_all_points_in_one_cell_and_duplicates():
    # heavy single cell: long lists go through the block sort
    rng = np.random.default_rng(1)
    pos = np.zeros((9000, 4), np.float32)
    pos[:, :3] = (0.5 + rng.random((9000, 3)) / 64).astype(np.float32)
    pos[100:200] = pos[50]                       # exact duplicates of point 50
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 5), 0, 0.03)
    off_o, ids_o = oracle_radius(scene)
    for method, walk in WALKS:
        off_g, ids_g = gpu_radius(scene, method=method, walk=walk)
        assert_csr_equal(off_g, ids_g, off_o, ids_o)
    assert np.diff(off_o).max() == 8999


def test_include_self_and_unsorted_lists():
    scene = synth.tiny_scene(8000, seed=5)
    off_o, ids_o = oracle_radius(scene, include_self=True)
    off_g, ids_g = gpu_radius(scene, include_self=True)
    assert_csr_equal(off_g, ids_g, off_o, ids_o)
    off_u, ids_u = gpu_radius(scene, include_self=True, sort=False)
    assert np.array_equal(off_u, off_o)
    for q in range(0, 8000, 7):
        assert np.array_equal(np.sort(ids_u[off_u[q]:off_u[q + 1]]), ids_o[off_o[q]:off_o[q + 1]])


def test_heavy_mixture_lists_sorted_and_exact():
    # Gaussian mixture on a coarse lattice: hundreds of neighbors per point
    pos = synth.gaussian_mixture_points(120_000, 21, n_comp=16, sigma=0.03)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 64, (6, 6, 6), 7, 1.5 / 64)
    off_g, ids_g = gpu_radius(scene)
    q = np.random.default_rng(0).choice(scene.n, 1500, replace=False)
    assert_sampled_equal(off_g, ids_g, scene, q)
    lens = np.diff(off_g)
    assert lens.max() > 500
    # symmetry of the whole relation
    rows = np.repeat(np.arange(scene.n), lens)
    fwd = rows.astype(np.int64) * scene.n + ids_g
    bwd = ids_g.astype(np.int64) * scene.n + rows
    assert np.array_equal(np.sort(fwd), np.sort(bwd))


def _sparse_cells_with_long_lists(scene, off_o, min_hits=64):
    """Queries in cells of at most two points whose lists exceed min_hits:
    their walks pass the per-thread candidate budget, so the warp-per-query
    kernels serve them."""
    c = np.floor((scene.pos[:, :3].astype(np.float64) - np.array(scene.origin)) / scene.cell_size)
    key = np.where((c < 0).any(1) | (c >= 2 ** np.array(scene.log2_cells)).any(1), -1,
                   c[:, 0] + 2 ** scene.log2_cells[0] * (c[:, 1] + 2 ** scene.log2_cells[1] * c[:, 2]))
    inside = key >= 0
    cnt = np.zeros(scene.n, dtype=np.int64)
    u, inv, k = np.unique(key[inside], return_inverse=True, return_counts=True)
    cnt[inside] = k[inv]
    return int(((cnt <= 2) & inside & (np.diff(off_o) > min_hits)).sum())


@pytest.mark.parametrize("mask", [7, 0])
def test_dense_light_queries_exact(mask):
    # sparse cells beside dense clusters: light queries with long lists; the
    # non-cyclic variant adds a cluster outside the region (queries outside
    # the region walk the bounding cube, their outside cell holds hundreds)
    pos = synth.gaussian_mixture_points(40_000, 31 + mask, n_comp=8, sigma=0.025)
    if mask == 0:
        out = synth.gaussian_mixture_points(600, 5, n_comp=1, sigma=0.004)
        out[:, 0] = 1.0 + 0.01 + out[:, 0] * 0.02
        pos = np.concatenate([pos, out]).astype(np.float32)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 5), mask, 1.5 / 32)
    off_o, ids_o = oracle_radius(scene)
    assert _sparse_cells_with_long_lists(scene, off_o) > 50
    off_g, ids_g = gpu_radius(scene)
    assert_csr_equal(off_g, ids_g, off_o, ids_o)
    off_s, ids_s = oracle_radius(scene, include_self=True)
    g = gpu_grid(scene)
    off_gs, ids_gs = gpu_radius(scene, include_self=True, grid=g)
    assert_csr_equal(off_gs, ids_gs, off_s, ids_s)
    off_u, ids_u = gpu_radius(scene, sort=False, grid=g)
    assert np.array_equal(off_u, off_o)
    for q in range(0, scene.n, 3):
        assert np.array_equal(np.sort(ids_u[off_u[q]:off_u[q + 1]]), ids_o[off_o[q]:off_o[q + 1]])


@pytest.mark.parametrize("mask", [7, 0])
def test_cells_split_into_index_slabs(mask):
    # ~15 points per cell and r = 2.9 cells: every cell has ~2.9k candidates,
    # more than the large cell kernel stages, so cells are split into slabs of
    # input indices whose hits concatenate into the sorted lists
    pos = synth.uniform_points(60_000, 41 + mask)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), mask, 2.9 / 16)
    off_o, ids_o = oracle_radius(scene)
    g = gpu_grid(scene)
    off_g, ids_g = gpu_radius(scene, grid=g)
    assert_csr_equal(off_g, ids_g, off_o, ids_o)
    assert np.diff(off_o).mean() > 1000
    if mask == 7:
        off_s, ids_s = oracle_radius(scene, include_self=True)
        off_gs, ids_gs = gpu_radius(scene, include_self=True, grid=g)
        assert_csr_equal(off_gs, ids_gs, off_s, ids_s)


def test_cells_split_into_three_or_more_slabs_sampled():
    pos = synth.uniform_points(100_000, 43)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), 7, 2.9 / 16)
    off_g, ids_g = gpu_radius(scene)
    q = np.random.default_rng(3).choice(scene.n, 800, replace=False)
    assert_sampled_equal(off_g, ids_g, scene, q)
    assert off_g[-1] % 2 == 0


@pytest.mark.parametrize("name", ["uniform_1m", "mixture_1m"])
def test_full_size_1m_configs_sampled(name):
    scene = synth.uniform_1m_scene() if name == "uniform_1m" else synth.mixture_1m_scene()
    g = gpu_grid(scene)
    for method, walk in WALKS:
        off, ids = g.query_radius(scene.r, method=method, walk=walk)
        g.sync()
        off_g, ids_g = off.cpu().numpy(), ids.cpu().numpy()
        if (method, walk) == WALKS[0]:
            q = np.random.default_rng(1).choice(scene.n, 1500, replace=False)
            assert_sampled_equal(off_g, ids_g, scene, q)
            ref = (off_g, ids_g)
        else:
            assert np.array_equal(off_g, ref[0]) and np.array_equal(ids_g, ref[1])
    # even number of directed pairs (symmetric relation)
    assert ref[0][-1] % 2 == 0


def test_capacity_overflow_and_invalid_inputs():
    scene = synth.tiny_scene(5000, seed=2)
    g = gpu_grid(scene)
    off = torch.empty(scene.n + 1, dtype=torch.int64, device="cuda")
    ids = torch.empty(10, dtype=torch.int32, device="cuda")
    with pytest.raises(_native.SIError) as ei:
        g.query_radius(scene.r, out_offsets=off, out_ids=ids)
    assert ei.value.status == _native.SI_ERR_CAPACITY
    # asynchronous overflow is reported by sync
    g.query_radius(scene.r, out_offsets=off, out_ids=ids, sync_total=False)
    with pytest.raises(_native.SIError) as ei:
        g.sync()
    assert ei.value.status == _native.SI_ERR_CAPACITY
    # radius beyond the tables
    with pytest.raises(_native.SIError):
        g.query_radius(scene.r * 2)
    # a cyclic coordinate outside its box is reported after the build
    bad = synth.uniform_points(100, 4)
    bad[3, 1] = np.float32(1.25)
    gc = Grid((0, 0, 0), 1 / 16, (4, 4, 4), 7, 0.1, 100)
    gc.build(to_dev(bad))
    with pytest.raises(_native.SIError) as ei:
        gc.sync()
    assert ei.value.status == _native.SI_ERR_INVALID

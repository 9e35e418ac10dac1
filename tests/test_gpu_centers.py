"""Parity of the radius and K-nearest queries from caller-given centers (the
general problem of Sec. I / Sec. II.A: a center and a radius) with the FP64
oracle: neighbor sets, counts and K-nearest order bit-exact; nothing is
excluded, so a center on top of a point finds it at distance 0."""
import numpy as np
import pytest
import torch

import oracle
from paper_cs_0608108_b300 import _native, synth

from gpu_helpers import assert_csr_equal, gpu_grid, oracle_radius, to_dev

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
WALKS = [("sphere", "classes"), ("sphere", "paper"), ("cube", "classes")]


def radius_centers(g, centers, r, method="sphere", walk="classes", sort=True):
    off, ids = g.query_radius(r, method=method, walk=walk, sort=sort, centers=to_dev(centers))
    g.sync()
    return off.cpu().numpy(), ids.cpu().numpy()


def oracle_centers(scene, centers, r=None):
    r = float(np.float32(scene.r if r is None else r))
    return oracle.radius(scene.pos, centers, scene.box, scene.cyclic_mask, r, None, threads=0)


def mixed_centers(scene, m, seed):
    """Uniform centers in the region, copies of points, centers on cell faces
    and corners, and duplicates."""
    rng = np.random.default_rng(seed)
    c = np.zeros((m, 4), np.float32)
    box = np.array(scene.box)
    c[:, :3] = (rng.random((m, 3)) * box + np.array(scene.origin)).astype(np.float32)
    k = m // 4
    c[:k] = scene.pos[rng.integers(0, scene.n, k)]                     # on top of points
    s = np.float32(scene.cell_size)
    cells = rng.integers(0, 1 << min(scene.log2_cells), (k, 3)).astype(np.float32)
    c[k:2 * k, :3] = cells * s + np.array(scene.origin, np.float32)   # cell corners
    c[2 * k:2 * k + 10] = c[0]                                          # duplicates
    return c


@pytest.mark.parametrize("mask", [7, 0, 5])
@pytest.mark.parametrize("r_cells", [0.45, 1.5, 2.7])
def test_random_centers_every_walk(mask, r_cells):
    pos = synth.uniform_points(20_000, 300 + mask)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), mask, r_cells / 16)
    c = mixed_centers(scene, 9000, mask)
    if mask != 7:   # centers outside the region on the non-cyclic axes
        for a in range(3):
            if not (mask >> a) & 1:
                c[a * 7:(a + 1) * 7, a] = np.float32(1.02 if a % 2 else -0.05)
    off_o, ids_o = oracle_centers(scene, c)
    g = gpu_grid(scene)
    for method, walk in WALKS:
        off_g, ids_g = radius_centers(g, c, scene.r, method, walk)
        assert_csr_equal(off_g, ids_g, off_o, ids_o)


def test_center_on_a_point_finds_it_at_distance_zero():
    scene = synth.Scene(synth.uniform_points(5000, 7), (0, 0, 0), 1 / 16, (4, 4, 4), 7, 1.5 / 16)
    c = scene.pos[[3, 3, 4000]].copy()
    off, ids = radius_centers(gpu_grid(scene), c, scene.r)
    for t, q in enumerate([3, 3, 4000]):
        assert q in ids[off[t]:off[t + 1]]
    off_o, ids_o = oracle_centers(scene, c)
    assert_csr_equal(off, ids, off_o, ids_o)


def test_clustered_points_long_lists_and_every_sort_path():
    # dense clusters: centers there are served a warp per center, and lists
    # run from a few ids to several thousand (warp and block sorts)
    clu = synth.gaussian_mixture_points(60_000, 21, n_comp=4, sigma=0.01)
    uni = synth.uniform_points(20_000, 22)
    pos = np.concatenate([clu, uni]).astype(np.float32)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 5), 7, 2.0 / 32)
    rng = np.random.default_rng(5)
    c = np.concatenate([clu[rng.integers(0, clu.shape[0], 3000)], synth.uniform_points(3000, 23)])
    c[:1000, :3] += rng.normal(0, 0.002, (1000, 3)).astype(np.float32)
    c[:, :3] = np.mod(c[:, :3], np.float32(1.0))
    c[:, :3] = np.where(c[:, :3] >= 1.0, np.float32(0.0), c[:, :3])
    off_o, ids_o = oracle_centers(scene, c)
    lens = np.diff(off_o)
    assert lens.max() > 2048 and (lens <= 32).any() and ((lens > 32) & (lens <= 512)).any()
    g = gpu_grid(scene)
    for method, walk in WALKS:
        off_g, ids_g = radius_centers(g, c, scene.r, method, walk)
        assert_csr_equal(off_g, ids_g, off_o, ids_o)
    # unsorted lists hold the same sets
    off_g, ids_g = radius_centers(g, c, scene.r, sort=False)
    assert np.array_equal(off_g, off_o)
    for t in range(0, c.shape[0], 7):
        assert np.array_equal(np.sort(ids_g[off_g[t]:off_g[t + 1]]), ids_o[off_o[t]:off_o[t + 1]])


def test_more_centers_than_points_and_regrowth():
    scene = synth.Scene(synth.uniform_points(3000, 31), (0, 0, 0), 1 / 16, (4, 4, 4), 3, 1.2 / 16)
    g = gpu_grid(scene)
    for m, seed in ((100, 1), (25_000, 2), (700, 3), (60_000, 4)):
        c = mixed_centers(scene, m, seed)
        off_g, ids_g = radius_centers(g, c, scene.r)
        assert_csr_equal(off_g, ids_g, *oracle_centers(scene, c))
    # the all-agents mode on the same grid is unaffected
    off, ids = g.query_radius(scene.r)
    g.sync()
    q = np.arange(scene.n)
    off_o, ids_o = oracle.radius(scene.pos, scene.pos, scene.box, scene.cyclic_mask, scene.r, q)
    assert_csr_equal(off.cpu().numpy(), ids.cpu().numpy(), off_o, ids_o)


def test_no_centers_and_empty_grid():
    scene = synth.Scene(synth.uniform_points(2000, 41), (0, 0, 0), 1 / 16, (4, 4, 4), 7, 1.5 / 16)
    g = gpu_grid(scene)
    off, ids = radius_centers(g, np.zeros((0, 4), np.float32), scene.r)
    assert off.tolist() == [0] and ids.size == 0
    empty = synth.Scene(np.zeros((0, 4), np.float32), (0, 0, 0), 1 / 16, (4, 4, 4), 7, 1.5 / 16)
    ge = gpu_grid(empty, capacity=16)
    c = mixed_centers(scene, 50, 1)
    off, ids = radius_centers(ge, c, scene.r)
    assert np.all(off == 0) and ids.size == 0
    ids, d2, cnt = ge.query_knn(4, r_max=scene.r, centers=to_dev(c))
    ge.sync()
    assert np.all(cnt.cpu().numpy() == 0) and np.all(ids.cpu().numpy() == -1)


def test_invalid_centers_get_empty_results_and_a_status():
    scene = synth.Scene(synth.uniform_points(4000, 51), (0, 0, 0), 1 / 16, (4, 4, 4), 3, 1.5 / 16)
    c = mixed_centers(scene, 400, 2)
    c[5, 0] = np.float32(1.25)      # outside the box on cyclic x
    c[9, 1] = np.float32(-0.5)      # outside on cyclic y
    c[11, 2] = np.float32(np.nan)   # non-finite
    c[13, 2] = np.float32(7.0)      # outside on non-cyclic z: a valid query
    bad = [5, 9, 11]
    good = np.setdiff1d(np.arange(c.shape[0]), bad)
    g = gpu_grid(scene)
    off, ids = g.query_radius(scene.r, centers=to_dev(c))
    with pytest.raises(_native.SIError) as e:
        g.sync()
    assert e.value.status == _native.SI_ERR_INVALID
    g.sync()    # the status is cleared once reported
    off, ids = off.cpu().numpy(), ids.cpu().numpy()
    assert all(off[b + 1] == off[b] for b in bad)
    off_o, ids_o = oracle_centers(scene, c[good])
    for t, q in enumerate(good):
        assert np.array_equal(ids[off[q]:off[q + 1]], ids_o[off_o[t]:off_o[t + 1]])
    ki, kd, kc = g.query_knn(6, r_max=scene.r, centers=to_dev(c))
    with pytest.raises(_native.SIError):
        g.sync()
    ki, kd, kc = ki.cpu().numpy(), kd.cpu().numpy(), kc.cpu().numpy()
    assert np.all(kc[bad] == 0) and np.all(ki[bad] == -1) and np.all(np.isinf(kd[bad]))
    oi, od, oc = oracle.knn(scene.pos, c[good], scene.box, scene.cyclic_mask, 6, scene.r)
    assert np.array_equal(kc[good], oc) and np.array_equal(ki[good], oi)


def check_knn(scene, c, k, r_max, ids, d2, cnt):
    if r_max is not None:
        r_max = float(np.float32(r_max))
    oi, od, oc = oracle.knn(scene.pos, c, scene.box, scene.cyclic_mask, k, r_max)
    assert np.array_equal(cnt, oc)
    assert np.array_equal(ids, oi)
    fin = np.isfinite(od)
    got = d2.astype(np.float64)
    assert np.all(np.isinf(got[~fin]))
    # the FP32 rounding of the canonical FP64 D2, exactly
    assert np.array_equal(d2[fin], od[fin].astype(np.float32))


@pytest.mark.parametrize("mask", [7, 3, 0])
@pytest.mark.parametrize("k", [1, 8, 64])
def test_knn_from_centers_within_r_max(mask, k):
    pos = synth.uniform_points(30_000, 60 + mask)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 5), mask, 4 / 32)
    c = mixed_centers(scene, 6000, k)
    if mask != 7:
        c[:12, 2] = np.float32(1.1)   # outside on non-cyclic z
    g = gpu_grid(scene, r_max=scene.r)
    ids, d2, cnt = g.query_knn(k, r_max=scene.r, centers=to_dev(c))
    g.sync()
    check_knn(scene, c, k, scene.r, ids.cpu().numpy(), d2.cpu().numpy(), cnt.cpu().numpy())


def test_knn_from_centers_unbounded_and_crowded():
    # unbounded r_max on a non-cyclic grid (per-thread kernel); and centers
    # in a tight cluster whose candidates overflow a warp's buffer
    scene = synth.tiny_scene()
    c = mixed_centers(scene, 5000, 9)
    g = gpu_grid(scene, r_max=float("inf"))
    ids, d2, cnt = g.query_knn(8, r_max=None, centers=to_dev(c))
    g.sync()
    check_knn(scene, c, 8, None, ids.cpu().numpy(), d2.cpu().numpy(), cnt.cpu().numpy())
    clu = synth.gaussian_mixture_points(2000, 13, n_comp=1, sigma=0.004)
    pos = np.concatenate([clu, synth.uniform_points(3000, 14)]).astype(np.float32)
    sc2 = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), 7, 2 / 16)
    c2 = np.concatenate([clu[::4], synth.uniform_points(500, 15)]).astype(np.float32)
    g2 = gpu_grid(sc2)
    for k in (16, 64):
        ids, d2, cnt = g2.query_knn(k, r_max=sc2.r, centers=to_dev(c2))
        g2.sync()
        check_knn(sc2, c2, k, sc2.r, ids.cpu().numpy(), d2.cpu().numpy(), cnt.cpu().numpy())


def test_full_size_uniform_1m_with_random_centers_sampled():
    # 1M points on the 128^3 cyclic lattice, 1M uniform random centers
    scene = synth.uniform_1m_scene()
    c = synth.uniform_points(1_000_000, 0x51D00099)
    g = gpu_grid(scene)
    off, ids = g.query_radius(scene.r, centers=to_dev(c))
    g.sync()
    off, ids = off.cpu().numpy(), ids.cpu().numpy()
    q = np.random.default_rng(3).choice(c.shape[0], 3000, replace=False)
    off_o, ids_o = oracle_centers(scene, c[q])
    for t, i in enumerate(q):
        assert np.array_equal(ids[off[i]:off[i + 1]], ids_o[off_o[t]:off_o[t + 1]])
    # mean list length: the expected points in a ball of r = 1.5 cells at
    # 0.477 points per cell (no self term)
    mean = (off[-1] / c.shape[0])
    expect = 4 / 3 * np.pi * 1.5 ** 3 * scene.n / 128 ** 3
    assert abs(mean - expect) < 0.02 * expect


# ---------------------------------------------------------------------------
# The non-empty list method (Sec. III.B, Sec. IV.A) and the volume comparison
# that switches to it.

def kernels_run(fn):
    """Names of the library kernels launched by fn()."""
    from paper_cs_0608108_b300 import _native as N
    import ctypes
    L = N.lib()
    L.si_kernel_timing_enable(1)
    buf = ctypes.create_string_buffer(1 << 16)
    L.si_kernel_timing_report(buf, len(buf))
    fn()
    L.si_kernel_timing_report(buf, len(buf))
    L.si_kernel_timing_enable(0)
    return {line.rsplit(" ", 2)[0] for line in buf.value.decode().splitlines() if line}


@pytest.mark.parametrize("mask", [7, 0, 6])
@pytest.mark.parametrize("include_self", [False, True])
def test_list_method_all_agents_exact(mask, include_self):
    pos = synth.uniform_points(9000, 500 + mask)
    pos[:6, 0] = np.float32(-0.2) if not (mask & 1) else pos[:6, 0]   # outside on a non-cyclic x
    pos[10:30] = pos[3]                                               # coincident points
    scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), mask, 2.3 / 16)
    g = gpu_grid(scene)
    off, ids = g.query_radius(scene.r, method="list", include_self=include_self)
    g.sync()
    q = np.arange(scene.n)
    off_o, ids_o = oracle.radius(scene.pos, scene.pos, scene.box, scene.cyclic_mask, scene.r,
                                 None if include_self else q)
    assert_csr_equal(off.cpu().numpy(), ids.cpu().numpy(), off_o, ids_o)


def test_list_method_from_centers_exact():
    scene = synth.Scene(synth.uniform_points(7000, 511), (0, 0, 0), 1 / 16, (4, 4, 4), 5, 3.1 / 16)
    c = mixed_centers(scene, 5000, 3)
    c[7, 1] = np.float32(-0.3)       # outside on the non-cyclic y
    c[8, 0] = np.float32(2.0)        # outside the cyclic x box: invalid
    g = gpu_grid(scene)
    off, ids = g.query_radius(scene.r, method="list", centers=to_dev(c))
    with pytest.raises(_native.SIError):
        g.sync()
    off, ids = off.cpu().numpy(), ids.cpu().numpy()
    assert off[9] == off[8]
    good = np.setdiff1d(np.arange(c.shape[0]), [8])
    off_o, ids_o = oracle_centers(scene, c[good])
    for t, i in enumerate(good):
        assert np.array_equal(ids[off[i]:off[i + 1]], ids_o[off_o[t]:off_o[t + 1]])


def test_method_weight_and_reversal_to_the_bin_lattice():
    # the Appendix's weighting factor and reversal distance: they change the
    # kernels a query runs, never its lists
    scene = synth.Scene(synth.uniform_points(30_000, 531), (0, 0, 0), 1 / 32, (5, 5, 5), 6, 1.2 / 32)
    off_o, ids_o = oracle_radius(scene)
    g = gpu_grid(scene)
    cases = [((0.0, 0.0), "k_radius_all_count"),            # weight 0: always the list
             ((float("inf"), 0.0), "k_radius_count"),       # never the list
             ((1.2, 2.0), "k_radius_count_cube"),           # r = 1.2 cells < 2: the cube scan
             ((1.2, 0.0), "k_radius_count")]                # the defaults
    for (w, cb), kernel in cases:
        g.set_method(w, cb)
        names = kernels_run(lambda: g.query_radius(scene.r))
        assert kernel in names, (w, cb, names)
        off, ids = g.query_radius(scene.r)
        g.sync()
        assert_csr_equal(off.cpu().numpy(), ids.cpu().numpy(), off_o, ids_o)
    with pytest.raises(_native.SIError):
        g.set_method(-1.0, 0.0)


def test_volume_comparison_picks_the_list_at_low_load_and_large_radius():
    # 64^3 cells for 20,480 points (load 0.08), r = 20 cells: the sphere holds
    # ~40k cells, more than the region has points
    far = synth.Scene(synth.uniform_points(20_480, 521), (0, 0, 0), 1 / 64, (6, 6, 6), 7, 20 / 64)
    g = gpu_grid(far)
    c = to_dev(mixed_centers(far, 3000, 4))
    names = kernels_run(lambda: g.query_radius(far.r, centers=c))
    assert "k_radius_all_count" in names and "k_radius_all_write" in names
    names = kernels_run(lambda: g.query_radius(far.r, centers=c, method="sphere_only"))
    assert "k_radius_all_count" not in names
    off_a, ids_a = radius_centers(g, c.cpu().numpy(), far.r)
    off_s, ids_s = radius_centers(g, c.cpu().numpy(), far.r, method="sphere_only")
    assert_csr_equal(off_a, ids_a, off_s, ids_s)
    # the 1M uniform configuration keeps the sphere
    near = synth.uniform_1m_scene()
    gn = gpu_grid(near)
    names = kernels_run(lambda: gn.query_radius(near.r))
    assert "k_radius_all_count" not in names

"""Parity of the CUDA K-nearest query with the FP64 oracle: ids (ordered by
(D2, index)) and counts bit-exact; the distances are the FP32 roundings of
the canonical FP64 D2, bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_cs_0608108_b300 import Grid, synth

from gpu_helpers import gpu_grid, to_dev

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def run_knn(scene, k, r_max):
    g = gpu_grid(scene, r_max=float("inf") if r_max is None else r_max)
    ids, d2, cnt = g.query_knn(k, r_max=r_max)
    g.sync()
    return ids.cpu().numpy(), d2.cpu().numpy(), cnt.cpu().numpy()


def check(scene, k, r_max, ids, d2, cnt, queries):
    if r_max is not None:
        r_max = float(np.float32(r_max))   # the radius the library receives
    oi, od, oc = oracle.knn(scene.pos, scene.pos[queries], scene.box, scene.cyclic_mask, k, r_max,
                            queries)
    assert np.array_equal(cnt[queries], oc)
    assert np.array_equal(ids[queries], oi)
    fin = np.isfinite(od)
    got = d2[queries].astype(np.float64)
    assert np.all(np.isinf(got[~fin]))
    # the FP32 rounding of the canonical FP64 D2, exactly
    assert np.array_equal(d2[queries][fin], od[fin].astype(np.float32))


def test_tiny_config_k8_unbounded_exact():
    scene = synth.tiny_scene()
    ids, d2, cnt = run_knn(scene, 8, None)
    check(scene, 8, None, ids, d2, cnt, np.arange(scene.n))
    assert np.all(cnt == 8)


@pytest.mark.parametrize("mask", [7, 3, 0, 4])
@pytest.mark.parametrize("k", [1, 5, 16, 40, 64])
def test_masks_and_k_within_r_max(mask, k):
    # 0.92 points per cell, 245 expected within r_max: the warp kernel's
    # first cut holds about K + 2 sqrt(K) + 4 candidates, so K = 40 sorts
    # 33-64 keys (two register slots) and K = 64 around 84 (65-96 in three
    # slots, 97-128 in four)
    pos = synth.uniform_points(30_000, 40 + mask)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 5), mask, 4 / 32)
    ids, d2, cnt = run_knn(scene, k, scene.r)
    check(scene, k, scene.r, ids, d2, cnt, np.arange(0, scene.n, 3))


def test_ties_on_a_coarse_lattice_broken_by_index():
    rng = np.random.default_rng(2)
    pos = np.zeros((20_000, 4), np.float32)
    pos[:, :3] = rng.integers(0, 64, size=(20_000, 3)) / 64.0
    scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), 7, 3 / 16)
    ids, d2, cnt = run_knn(scene, 12, scene.r)
    check(scene, 12, scene.r, ids, d2, cnt, np.arange(scene.n))


def _float32_midpoints(od):
    """How many FP64 values lie exactly halfway between two FP32 values."""
    f = od.astype(np.float32)
    lo = f.astype(np.float64)
    nb = np.nextafter(f, np.where(od > lo, np.float32(np.inf), np.float32(-np.inf))).astype(np.float64)
    return int(np.sum((od != lo) & (2.0 * od == lo + nb)))


@pytest.mark.parametrize("mask", [7, 0])
def test_distances_at_float32_midpoints(mask):
    """Coordinates on a 2^-16 grid: squared distances carry about 27
    significant bits, so many canonical values fall exactly halfway between
    two FP32 values (and many more within a few units of the 2^-40 margin),
    where the FP32 form of the rounding hands over to FP64; ties-to-even
    must come out as the FP64 conversion does."""
    rng = np.random.default_rng(11 + mask)
    pos = np.zeros((20_000, 4), np.float32)
    pos[:, :3] = rng.integers(0, 1 << 16, size=(20_000, 3)) / float(1 << 16)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 5), mask, 3 / 32)
    ids, d2, cnt = run_knn(scene, 16, scene.r)
    q = np.arange(scene.n)
    check(scene, 16, scene.r, ids, d2, cnt, q)
    _, od, _ = oracle.knn(scene.pos, scene.pos, scene.box, scene.cyclic_mask, 16, float(np.float32(scene.r)), q)
    assert _float32_midpoints(od[np.isfinite(od)]) > 1000


def test_duplicates_and_points_outside_region():
    pos = synth.uniform_points(8000, 8)
    pos[100:140] = pos[7]                  # 40 copies of point 7: distance-0 ties
    pos[:20, 2] = np.float32(1.3)          # outside on a non-cyclic z
    scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), 3, 2 / 16)
    ids, d2, cnt = run_knn(scene, 16, scene.r)
    check(scene, 16, scene.r, ids, d2, cnt, np.arange(scene.n))


@pytest.mark.parametrize("k", [16, 64])
def test_full_size_4m_config_sampled(k):
    scene = synth.knn_4m_scene()
    ids, d2, cnt = run_knn(scene, k, scene.r)
    q = np.random.default_rng(k).choice(scene.n, 600, replace=False)
    check(scene, k, scene.r, ids, d2, cnt, q)
    if k == 64:
        # about half the points have fewer than 64 neighbors within 4 cells
        assert 0.3 < (cnt < 64).mean() < 0.7


def test_crowded_queries_overflowing_the_warp_buffer():
    # a tight cluster: its points have ~2000 candidates within r_max, more
    # than a warp buffers, and are served by the per-thread kernel instead
    clu = synth.gaussian_mixture_points(2000, 13, n_comp=1, sigma=0.004)
    uni = synth.uniform_points(3000, 14)
    pos = np.concatenate([clu, uni]).astype(np.float32)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), 7, 2 / 16)
    for k in (16, 64):
        ids, d2, cnt = run_knn(scene, k, scene.r)
        check(scene, k, scene.r, ids, d2, cnt, np.arange(scene.n))


@pytest.mark.parametrize("k", [1, 8, 16, 40])
@pytest.mark.parametrize("mask", [7, 0])
def test_include_self_through_both_kernels(k, mask):
    # K <= 16 runs the thread-per-query kernel, K = 40 the warp kernel; the
    # query's own point comes first, at distance 0
    pos = synth.uniform_points(20_000, 60 + mask)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 5), mask, 3 / 32)
    g = gpu_grid(scene)
    ids, d2, cnt = g.query_knn(k, r_max=scene.r, include_self=True)
    g.sync()
    ids, d2, cnt = ids.cpu().numpy(), d2.cpu().numpy(), cnt.cpu().numpy()
    q = np.arange(scene.n)
    oi, od, oc = oracle.knn(scene.pos, scene.pos, scene.box, mask, k, float(np.float32(scene.r)), None)
    assert np.array_equal(cnt, oc) and np.array_equal(ids, oi)
    fin = np.isfinite(od)
    assert np.array_equal(d2[fin], od[fin].astype(np.float32))
    assert np.all(ids[:, 0] == q) and np.all(d2[:, 0] == 0.0)


@pytest.mark.parametrize("k", [1, 16, 64])
@pytest.mark.parametrize("mask", [7, 0])
def test_bin_lattice_walk_gives_the_same_results(k, mask):
    # the K-nearest query through the bin lattice (every cell of the bounding
    # cube of the r_max sphere): the oracle's ids, counts and distances
    pos = synth.uniform_points(20_000, 80 + mask)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 5), mask, 3 / 32)
    g = gpu_grid(scene)
    ids, d2, cnt = g.query_knn(k, r_max=scene.r, method="cube")
    g.sync()
    check(scene, k, scene.r, ids.cpu().numpy(), d2.cpu().numpy(), cnt.cpu().numpy(), np.arange(scene.n))


def test_knn_reversal_distance_switches_to_the_bin_lattice():
    from test_gpu_centers import kernels_run
    pos = synth.uniform_points(10_000, 91)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 5), 7, 2 / 32)
    g = gpu_grid(scene)
    ref = [t.cpu().numpy() for t in g.query_knn(8, r_max=scene.r)]
    assert "k_knn_cube" not in kernels_run(lambda: g.query_knn(8, r_max=scene.r))
    g.set_method(knn_cube_below=3.0)        # r_max = 2 cells < 3: the bin lattice
    assert "k_knn_cube" in kernels_run(lambda: g.query_knn(8, r_max=scene.r))
    got = [t.cpu().numpy() for t in g.query_knn(8, r_max=scene.r)]
    assert all(np.array_equal(a, b) for a, b in zip(ref, got))


def test_fast_distances_within_their_bound():
    # SI_FAST_D2: the same ids and counts, the kernel's FP32 squared distance
    # within 12u D2 + 16u L sqrt(D2) of the canonical D2
    pos = synth.uniform_points(30_000, 77)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 5), 3, 4 / 32)
    g = gpu_grid(scene)
    q = np.arange(0, scene.n, 5)
    for k in (16, 40):   # the thread-per-query kernel, then the warp kernel
        ids, d2, cnt = g.query_knn(k, r_max=scene.r, fast_d2=True)
        g.sync()
        oi, od, oc = oracle.knn(scene.pos, scene.pos[q], scene.box, 3, k, float(np.float32(scene.r)), q)
        assert np.array_equal(cnt.cpu().numpy()[q], oc) and np.array_equal(ids.cpu().numpy()[q], oi)
        got = d2.cpu().numpy()[q].astype(np.float64)
        fin = np.isfinite(od)
        assert np.all(np.isinf(got[~fin]))
        L = max(scene.box)
        assert np.all(np.abs(got[fin] - od[fin]) <= 12 * U * od[fin] + 16 * U * L * np.sqrt(od[fin]) + 1e-30)

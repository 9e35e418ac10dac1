"""Parity at the limits of the descriptor and of the method: the largest
lattice (2^27 cells), the largest radius a cyclic axis allows, r = 0
(coincident points only), every point at one position, and K above the
number of points."""
import numpy as np
import pytest
import torch

import oracle
from paper_cs_0608108_b300 import Grid, synth

from gpu_helpers import assert_csr_equal, gpu_grid, oracle_radius, to_dev

pytestmark = pytest.mark.gpu

METHODS = ["sphere", "sphere_only", "list", "cube"]


def test_largest_lattice_sampled():
    # 1024 x 1024 x 128 cells (sum of log2 = 27), cyclic, r = 1.5 cells
    n = 400_000
    pos = synth.uniform_points(n, 81, box=(1.0, 1.0, 0.125))
    scene = synth.Scene(pos, (0, 0, 0), 1 / 1024, (10, 10, 7), 7, 1.5 / 1024)
    g = gpu_grid(scene)
    assert g.info()["n_cells"] == (1 << 27) + 1
    off, ids = g.query_radius(scene.r)
    g.sync()
    off, ids = off.cpu().numpy(), ids.cpu().numpy()
    q = np.random.default_rng(8).choice(n, 2000, replace=False)
    off_o, ids_o = oracle_radius(scene, queries=q)
    for t, i in enumerate(q):
        assert np.array_equal(ids[off[i]:off[i + 1]], ids_o[off_o[t]:off_o[t + 1]])
    ki, kd, kc = g.query_knn(8, r_max=scene.r)
    g.sync()
    oi, od, oc = oracle.knn(scene.pos, scene.pos[q], scene.box, 7, 8, scene.r, q)
    assert np.array_equal(kc.cpu().numpy()[q], oc) and np.array_equal(ki.cpu().numpy()[q], oi)


def test_largest_cyclic_radius_every_method():
    # on 16 cyclic cells the tables allow floor(d) <= 6: d = 6.9 cells
    pos = synth.uniform_points(8000, 82)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), 7, 6.9 / 16)
    off_o, ids_o = oracle_radius(scene)
    g = gpu_grid(scene)
    for method in METHODS:
        off, ids = g.query_radius(scene.r, method=method)
        g.sync()
        assert_csr_equal(off.cpu().numpy(), ids.cpu().numpy(), off_o, ids_o)
    # one cell further is rejected
    with pytest.raises(Exception):
        Grid((0, 0, 0), 1 / 16, (4, 4, 4), 7, 7.0 / 16, 10)


@pytest.mark.parametrize("mask", [7, 0])
def test_zero_radius_finds_coincident_points_only(mask):
    pos = synth.uniform_points(6000, 83 + mask)
    pos[100:140] = pos[7]            # 41 points at one position
    pos[500:503] = pos[499]          # 4 at another
    scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), mask, 0.0)
    g = gpu_grid(scene, r_max=1 / 16)
    off_o, ids_o = oracle_radius(scene, r=0.0)
    for method in METHODS:
        off, ids = g.query_radius(0.0, method=method)
        g.sync()
        assert_csr_equal(off.cpu().numpy(), ids.cpu().numpy(), off_o, ids_o)
    lens = np.diff(off_o)
    assert lens[7] == 40 and lens[499] == 3 and lens[0] == 0


def test_every_point_at_one_position():
    pos = np.tile(synth.uniform_points(1, 84), (3000, 1))
    scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), 7, 0.5 / 16)
    g = gpu_grid(scene)
    for method in METHODS:
        off, ids = g.query_radius(scene.r, method=method)
        g.sync()
        off, ids = off.cpu().numpy(), ids.cpu().numpy()
        assert np.all(np.diff(off) == 2999)
        for i in (0, 1234, 2999):
            assert np.array_equal(ids[off[i]:off[i + 1]], np.delete(np.arange(3000), i))
    ki, kd, kc = g.query_knn(5, r_max=scene.r)
    g.sync()
    ki = ki.cpu().numpy()
    assert np.all(kc.cpu().numpy() == 5)
    assert np.array_equal(ki[0], [1, 2, 3, 4, 5]) and np.array_equal(ki[3], [0, 1, 2, 4, 5])


def test_k_above_the_number_of_points():
    pos = synth.uniform_points(10, 85)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 8, (3, 3, 3), 0, 1.0)
    g = gpu_grid(scene, r_max=float("inf"))
    ids, d2, cnt = g.query_knn(64, r_max=None)
    g.sync()
    oi, od, oc = oracle.knn(scene.pos, scene.pos, scene.box, 0, 64, None, np.arange(10))
    assert np.all(cnt.cpu().numpy() == 9) and np.array_equal(ids.cpu().numpy(), oi)
    assert np.all(np.isinf(d2.cpu().numpy()[:, 9:]))


def test_caller_output_buffers_are_checked_before_the_call():
    scene = synth.tiny_scene(2000, seed=3)
    g = gpu_grid(scene)
    small = torch.empty(10, dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        g.query_radius(scene.r, out_offsets=small)
    with pytest.raises(ValueError):
        g.query_radius(scene.r, out_offsets=torch.empty(scene.n + 1, dtype=torch.int32, device="cuda"))
    ids = torch.empty((scene.n, 4), dtype=torch.int32, device="cuda")
    cnt = torch.empty(scene.n, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        g.query_knn(8, r_max=scene.r, out=(ids, None, cnt))       # room for 4 per query, not 8
    with pytest.raises(ValueError):
        g.neighbor_reduce(scene.r, energy=torch.empty(1, dtype=torch.float32, device="cuda"))
    off, lst = g.query_radius(scene.r)                             # the grid is still usable
    g.sync()
    assert_csr_equal(off.cpu().numpy(), lst.cpu().numpy(), *oracle_radius(scene))

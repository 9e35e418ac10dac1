"""Parity of the stacked-plane walk (Sec. V: circle-indexed z-planes, each
skipped when empty, taken as its point list when sparse, else walked by
rows) with the FP64 oracle: lists bit-exact for every cyclic mask, on
uniform points, on points concentrated on a terrain surface with a few
flying objects, and from caller-given centers."""
import numpy as np
import pytest

import oracle
from paper_cs_0608108_b300 import synth

from gpu_helpers import assert_csr_equal, gpu_grid, gpu_radius, oracle_radius, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mask", [0, 1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("r_cells", [0.45, 1.5, 3.7])
def test_planes_walk_uniform_every_mask(mask, r_cells):
    pos = synth.uniform_points(12_000, 700 + mask)
    for a in range(3):                       # points outside on the non-cyclic axes
        if not (mask >> a) & 1:
            pos[a * 5:(a + 1) * 5, a] = np.float32(1.07 if a % 2 else -0.03)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), mask, r_cells / 16)
    off_g, ids_g = gpu_radius(scene, walk="planes")
    assert_csr_equal(off_g, ids_g, *oracle_radius(scene))


@pytest.mark.parametrize("mask", [3, 7])
def test_planes_walk_terrain_with_flying_objects(mask):
    # most planes empty, two or three dense, a few holding a flying object
    pos = synth.terrain_points(40_000, 71, flying=0.003)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 64, (6, 6, 6), mask, 2.5 / 64)
    off_o, ids_o = oracle_radius(scene)
    g = gpu_grid(scene)
    for include_self in (False, True):
        off, ids = g.query_radius(scene.r, walk="planes", include_self=include_self)
        g.sync()
        ref = oracle_radius(scene, include_self=True) if include_self else (off_o, ids_o)
        assert_csr_equal(off.cpu().numpy(), ids.cpu().numpy(), *ref)
    off, ids = g.query_radius(scene.r, walk="planes", sort=False)
    g.sync()
    off, ids = off.cpu().numpy(), ids.cpu().numpy()
    assert np.array_equal(off, off_o)
    for q in range(0, scene.n, 97):
        assert np.array_equal(np.sort(ids[off[q]:off[q + 1]]), ids_o[off_o[q]:off_o[q + 1]])


def test_planes_walk_long_lists_and_centers():
    # a dense sheet: lists of hundreds of ids (the sorting paths), and
    # caller-given centers above, on and below it
    pos = synth.terrain_points(60_000, 72, flying=0.01, amp=0.002)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 5), 3, 2.0 / 32)
    g = gpu_grid(scene)
    off, ids = g.query_radius(scene.r, walk="planes")
    g.sync()
    off_o, ids_o = oracle_radius(scene)
    assert_csr_equal(off.cpu().numpy(), ids.cpu().numpy(), off_o, ids_o)
    assert np.diff(off_o).max() > 128
    cen = synth.uniform_points(5000, 73)
    cen[:2000, 2] = np.float32(0.5)
    cen[2000:2100, 2] = np.float32(1.4)       # outside on the non-cyclic z
    off_c, ids_c = g.query_radius(scene.r, walk="planes", centers=to_dev(cen))
    g.sync()
    off_co, ids_co = oracle.radius(scene.pos, cen, scene.box, scene.cyclic_mask, scene.r, None)
    assert_csr_equal(off_c.cpu().numpy(), ids_c.cpu().numpy(), off_co, ids_co)

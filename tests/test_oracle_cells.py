"""The CPU cell walks of oracle/cells.c (cube scan, spherical index with the
Eq. 1 cell test) give the brute force's lists exactly: every cyclic mask,
points outside the region on non-cyclic axes, radii across cell sizes, a
non-power-of-two cell side with an offset origin."""
import numpy as np
import pytest

import oracle
from paper_cs_0608108_b300 import synth


def brute(scene, r):
    return oracle.radius(scene.pos, scene.pos, scene.box, scene.cyclic_mask, r, np.arange(scene.n))


@pytest.mark.parametrize("mask", range(8))
@pytest.mark.parametrize("r_cells", [0.45, 1.5, 2.7])
def test_cell_walks_equal_brute_force(mask, r_cells):
    pos = synth.uniform_points(3000, 500 + mask)
    for a in range(3):
        if not (mask >> a) & 1:
            pos[a * 4:(a + 1) * 4, a] = np.float32(1.07 if a % 2 else -0.03)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), mask, r_cells / 16)
    r = float(np.float32(scene.r))
    off_b, ids_b = brute(scene, r)
    for method in ("sphere", "cube"):
        off_c, ids_c = oracle.cells_radius(scene.pos, scene.origin, scene.cell_size, scene.log2_cells,
                                           scene.cyclic_mask, r, method=method)
        assert np.array_equal(off_c, off_b) and np.array_equal(ids_c, ids_b), method


def test_offset_origin_and_sampled_queries():
    base = synth.uniform_points(4000, 77, box=(5.92, 5.92, 5.92), origin=(-2.0, 1.0, 3.0))
    scene = synth.Scene(base, (-2.0, 1.0, 3.0), 0.37, (4, 4, 4), 5, 0.37 * 1.7)
    r = float(np.float32(scene.r))
    q = np.arange(0, scene.n, 7)
    off_b, ids_b = oracle.radius(scene.pos, scene.pos[q], scene.box, scene.cyclic_mask, r, q)
    for method in ("sphere", "cube"):
        off_c, ids_c = oracle.cells_radius(scene.pos, scene.origin, scene.cell_size, scene.log2_cells,
                                           scene.cyclic_mask, r, queries=q, method=method)
        assert np.array_equal(off_c, off_b) and np.array_equal(ids_c, ids_b), method


def test_radius_wrapping_a_cyclic_axis_is_refused():
    scene = synth.Scene(synth.uniform_points(100, 3), (0, 0, 0), 1 / 4, (2, 2, 2), 7, 0.3)
    with pytest.raises(ValueError):
        oracle.cells_radius(scene.pos, scene.origin, scene.cell_size, scene.log2_cells, 7, 0.3)

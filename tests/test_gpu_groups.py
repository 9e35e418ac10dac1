"""Parity of the grouped heavy-cell path (aligned 2x2x2 groups of crowded
cells sharing one candidate gather and id sort) with the FP64 oracle and
with every crowded cell served on its own: neighbor sets bit-exact."""
import numpy as np
import pytest

from paper_cs_0608108_b300 import synth

from gpu_helpers import assert_csr_equal, assert_sampled_equal, gpu_grid, gpu_radius, oracle_radius

pytestmark = pytest.mark.gpu


def _clusters_on_the_faces(n, seed, sigma):
    """Gaussian clusters, half of them centred on the box faces and corners,
    so that groups of crowded cells meet the cyclic wrap on every axis."""
    pos = synth.gaussian_mixture_points(n, seed, n_comp=12, sigma=sigma)
    k = np.arange(n) % 4
    # shift a quarter of the points onto a corner cluster and one onto each face
    pos[k == 1, 0] = np.mod(pos[k == 1, 0] - pos[k == 1, 0].mean() + 0.999, 1.0).astype(np.float32)
    pos[k == 2, 1] = np.mod(pos[k == 2, 1] - pos[k == 2, 1].mean() + 0.001, 1.0).astype(np.float32)
    pos[k == 3, 2] = np.mod(pos[k == 3, 2] - pos[k == 3, 2].mean(), 1.0).astype(np.float32)
    return pos


@pytest.mark.parametrize("mask", [7, 0, 3, 5])
def test_groups_exact_every_mask(mask):
    pos = _clusters_on_the_faces(60_000, 50 + mask, 0.03)
    if mask != 7:   # points outside the region on the non-cyclic axes
        for a in range(3):
            if not (mask >> a) & 1:
                pos[a * 40:(a + 1) * 40, a] = np.float32(1.01 + 0.001 * a)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 5), mask, 1.5 / 32)
    off_o, ids_o = oracle_radius(scene)
    g = gpu_grid(scene)
    off_g, ids_g = gpu_radius(scene, grid=g)
    assert_csr_equal(off_g, ids_g, off_o, ids_o)
    off = g.query_radius(scene.r, groups=False)
    g.sync()
    assert np.array_equal(off[0].cpu().numpy(), off_o) and np.array_equal(off[1].cpu().numpy(), ids_o)
    off_s, ids_s = oracle_radius(scene, include_self=True)
    off_gs, ids_gs = gpu_radius(scene, include_self=True, grid=g)
    assert_csr_equal(off_gs, ids_gs, off_s, ids_s)


def test_groups_with_crowded_and_overflowing_cells():
    # very tight clusters: cells with more than a block's queries and groups
    # whose candidate union exceeds a block go to the large per-cell kernel
    pos = synth.gaussian_mixture_points(80_000, 61, n_comp=6, sigma=0.02)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 64, (6, 6, 6), 7, 1.2 / 64)
    g = gpu_grid(scene)
    off_g, ids_g = gpu_radius(scene, grid=g)
    q = np.random.default_rng(4).choice(scene.n, 1200, replace=False)
    assert_sampled_equal(off_g, ids_g, scene, q)
    off = g.query_radius(scene.r, groups=False)
    g.sync()
    assert np.array_equal(off[0].cpu().numpy(), off_g) and np.array_equal(off[1].cpu().numpy(), ids_g)
    counts = np.bincount(np.floor(scene.pos[:, :3].astype(np.float64) * 64).astype(np.int64) @ [1, 64, 4096],
                         minlength=64 ** 3)
    assert counts.max() > 128


@pytest.mark.parametrize("log2", [(2, 2, 2), (3, 3, 3), (5, 2, 5)])
def test_small_lattices_fall_back_to_single_cells(log2):
    # lattices too small for a group's rows (fewer than 6 cells on an axis
    # at this radius): every crowded cell on its own; 8 cells per axis is the
    # smallest lattice with groups
    box = tuple(float(np.float32(0.05 * (1 << w))) for w in log2)
    pos = synth.gaussian_mixture_points(20_000, 71, n_comp=3, sigma=0.02)
    pos[:, :3] = (pos[:, :3] * np.array(box, dtype=np.float32)).astype(np.float32)
    pos[:, :3] = np.minimum(pos[:, :3], np.nextafter(np.array(box, dtype=np.float32), 0))
    scene = synth.Scene(pos, (0, 0, 0), 0.05, log2, 0, 0.05 * 1.4)
    off_o, ids_o = oracle_radius(scene)
    off_g, ids_g = gpu_radius(scene)
    assert_csr_equal(off_g, ids_g, off_o, ids_o)

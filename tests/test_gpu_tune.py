"""Discretization tuning (Sec. IV.A, Fig. 9 and 10): every valid candidate
lattice is timed, invalid ones are reported as +inf, the fastest is named."""
import math

import numpy as np
import pytest
import torch

from paper_cs_0608108_b300 import _native, synth, tune_lattice

from gpu_helpers import assert_csr_equal, gpu_grid, oracle_radius, to_dev

pytestmark = pytest.mark.gpu


def test_radius_candidates_all_valid():
    pos = to_dev(synth.uniform_points(65_536, 71))
    shifts = [-2, -1, 0, 1, 2]
    ms, best = tune_lattice((0, 0, 0), 1 / 16, (4, 4, 4), 7, pos, 1.5 / 16, shifts, reps=3)
    assert len(ms) == 5 and all(math.isfinite(t) and t > 0 for t in ms)
    assert best == int(np.argmin(ms))


def test_invalid_candidates_are_infinite():
    pos = to_dev(synth.uniform_points(20_000, 72))
    # r = 5 cells of 16^3: 8^3 is valid, 4^3 would wrap its tables, 2^3 is no lattice
    ms, best = tune_lattice((0, 0, 0), 1 / 16, (4, 4, 4), 7, pos, 5 / 16, [-3, -2, -1, 0], reps=2)
    assert math.isinf(ms[0]) and math.isinf(ms[1])
    assert math.isfinite(ms[2]) and math.isfinite(ms[3]) and best in (2, 3)
    with pytest.raises(_native.SIError):
        tune_lattice((0, 0, 0), 1 / 16, (4, 4, 4), 7, pos, 5 / 16, [-3, -2], reps=2)


def test_knn_and_centers_and_the_grid_afterwards():
    scene = synth.Scene(synth.uniform_points(40_000, 73), (0, 0, 0), 1 / 32, (5, 5, 5), 0, 2 / 32)
    pos = to_dev(scene.pos)
    c = to_dev(synth.uniform_points(30_000, 74))
    ms, best = tune_lattice(scene.origin, scene.cell_size, scene.log2_cells, 0, pos, scene.r, [-1, 0, 1],
                            centers=c, k=1, reps=3)
    assert all(math.isfinite(t) for t in ms) and best == int(np.argmin(ms))
    ms, best = tune_lattice(scene.origin, scene.cell_size, scene.log2_cells, 0, pos, scene.r, [-1, 0, 1],
                            centers=c, k=0, reps=3)
    assert all(math.isfinite(t) for t in ms)
    # the library is in a clean state: a fresh grid answers exactly
    off, ids = gpu_grid(scene).query_radius(scene.r)
    torch.cuda.synchronize()
    assert_csr_equal(off.cpu().numpy(), ids.cpu().numpy(), *oracle_radius(scene))

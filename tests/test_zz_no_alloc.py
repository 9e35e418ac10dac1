"""GPU test of si_neighbor_energy_noalloc, the entry point for callers that
cannot allocate device memory (frameworks that own every allocation, fixed
memory budgets, real-time steps).  Its scratch is a static device array
shared by all calls, so the test makes several calls in a row on different
inputs and checks each against the grid-based si_neighbor_reduce.

This file is collected last on purpose: a failure here leaves every other
test already run."""
import ctypes

import numpy as np
import pytest
import torch

from paper_cs_0608108_b300 import Grid, _native, make_desc, synth

pytestmark = pytest.mark.gpu

TOL = 1e-4      # relative energy tolerance of the reduction tests


def grid_energy(scene):
    g = Grid(scene.origin, scene.cell_size, scene.log2_cells, scene.cyclic_mask, scene.r, scene.n)
    g.build(torch.from_numpy(scene.pos).cuda())
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    g.neighbor_reduce(scene.r, energy=e)
    g.sync()
    return float(e.item())


def noalloc_energy(scene):
    lib = _native.lib()
    desc = make_desc(scene.origin, scene.cell_size, scene.log2_cells, scene.cyclic_mask, scene.r)
    pos = torch.from_numpy(scene.pos).cuda()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _native.check(lib.si_neighbor_energy_noalloc(ctypes.byref(desc), ctypes.c_void_p(pos.data_ptr()),
                                                 scene.n, float(scene.r),
                                                 ctypes.c_void_p(out.data_ptr()), st),
                  "si_neighbor_energy_noalloc")
    torch.cuda.synchronize()
    return float(out.item())


def test_noalloc_energy_matches_grid_path_on_calls_in_a_row():
    a = synth.Scene(synth.uniform_points(40_000, 31), (0, 0, 0), 1 / 32, (5, 5, 5), 7, 1.5 / 32)
    pb = synth.uniform_points(9_000, 32)
    pb[:5, 2] = np.float32(1.2)            # outside on a non-cyclic z
    b = synth.Scene(pb, (0, 0, 0), 1 / 16, (4, 4, 4), 3, 2.2 / 16)
    for scene in (a, b, a):
        want = grid_energy(scene)
        got = noalloc_energy(scene)
        assert want > 0
        assert abs(got - want) <= TOL * want


def test_noalloc_limits_and_invalid_points():
    lib = _native.lib()
    big = synth.Scene(synth.uniform_points(70_000, 1), (0, 0, 0), 1 / 32, (5, 5, 5), 7, 0.04)
    desc = make_desc(big.origin, big.cell_size, big.log2_cells, 7, big.r)
    pos = torch.from_numpy(big.pos).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.si_neighbor_energy_noalloc(ctypes.byref(desc), ctypes.c_void_p(pos.data_ptr()), big.n,
                                          0.04, ctypes.c_void_p(out.data_ptr()), st) == _native.SI_ERR_INVALID
    desc = make_desc((0, 0, 0), 1 / 64, (6, 6, 6), 7, 0.04)      # 2^18 cells
    assert lib.si_neighbor_energy_noalloc(ctypes.byref(desc), ctypes.c_void_p(pos.data_ptr()), 1000,
                                          0.04, ctypes.c_void_p(out.data_ptr()), st) == _native.SI_ERR_INVALID
    bad = synth.uniform_points(500, 2)
    bad[7, 0] = np.float32(1.5)            # outside a cyclic x: flagged, energy NaN
    scene = synth.Scene(bad, (0, 0, 0), 1 / 16, (4, 4, 4), 7, 0.1)
    assert np.isnan(noalloc_energy(scene))
    good = synth.Scene(synth.uniform_points(500, 2), (0, 0, 0), 1 / 16, (4, 4, 4), 7, 0.1)
    assert abs(noalloc_energy(good) - grid_energy(good)) <= TOL * grid_energy(good)


def test_noalloc_at_its_limits():
    # exactly the maxima: 65,536 points on a 2^16-cell lattice (5 + 5 + 6),
    # which fills every scratch region to its computed end; two calls in a row
    pos = synth.uniform_points(65_536, 33, box=(1.0, 1.0, 2.0))
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 6), 7, 1.4 / 32)
    want = grid_energy(scene)
    for _ in range(2):
        got = noalloc_energy(scene)
        assert want > 0 and abs(got - want) <= TOL * want

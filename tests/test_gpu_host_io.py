"""The end-to-end entry point with host buffers (si_query_radius_host): the
CSR result copied back to host memory equals the oracle's, from pageable and
page-locked host memory, and an ids buffer that is too small is refused
with nothing written."""
import numpy as np
import pytest
import torch

from paper_cs_0608108_b300 import Grid, synth, _native

from gpu_helpers import oracle_radius

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("mask", [7, 0])
def test_host_buffers_equal_the_oracle(pinned, mask):
    pos = synth.uniform_points(20_000, 900 + mask)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 5), mask, 1.5 / 32)
    off_o, ids_o = oracle_radius(scene)
    g = Grid.for_scene(scene)
    h_pos = torch.from_numpy(scene.pos)
    h_off = torch.zeros(scene.n + 1, dtype=torch.int64)
    h_ids = torch.zeros(int(off_o[-1]) + 100, dtype=torch.int32)
    if pinned:
        h_pos, h_off, h_ids = h_pos.pin_memory(), h_off.pin_memory(), h_ids.pin_memory()
    for _ in range(2):   # the second call reuses the grid's device buffers
        total = g.query_radius_host(h_pos, scene.r, h_off, h_ids)
        assert total == off_o[-1]
        assert np.array_equal(h_off.numpy(), off_o)
        assert np.array_equal(h_ids.numpy()[:total], ids_o)


def test_host_ids_buffer_too_small_is_refused():
    scene = synth.Scene(synth.uniform_points(5000, 17), (0, 0, 0), 1 / 16, (4, 4, 4), 7, 1.5 / 16)
    g = Grid.for_scene(scene)
    h_pos = torch.from_numpy(scene.pos)
    h_off = torch.zeros(scene.n + 1, dtype=torch.int64)
    h_ids = torch.full((10,), -7, dtype=torch.int32)
    with pytest.raises(_native.SIError):
        g.query_radius_host(h_pos, scene.r, h_off, h_ids)
    assert torch.all(h_ids == -7)
    # a large enough buffer then succeeds on the same grid
    off_o, ids_o = oracle_radius(scene)
    h_ids = torch.zeros(int(off_o[-1]), dtype=torch.int32)
    total = g.query_radius_host(h_pos, scene.r, h_off, h_ids)
    assert total == off_o[-1] and np.array_equal(h_ids.numpy(), ids_o)

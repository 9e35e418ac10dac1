"""The single-scene calls are capturable: once a grid's tables and buffers
are sized, si_grid_build + si_query_radius (walk or list method) issue no
host synchronisation, so a step captured in a CUDA graph and replayed gives
the eager results, also after the points are moved in place."""
import numpy as np
import pytest
import torch

from paper_cs_0608108_b300 import Grid, synth

from gpu_helpers import assert_csr_equal, oracle_radius

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", ["sphere", "list"])
def test_captured_build_and_query_replays_exactly(method):
    clu = synth.gaussian_mixture_points(30_000, 91, n_comp=8, sigma=0.02)
    scene = synth.Scene(np.concatenate([clu, synth.uniform_points(30_000, 92)]), (0, 0, 0), 1 / 32, (5, 5, 5), 7,
                        1.5 / 32)
    pos = torch.from_numpy(scene.pos).cuda()
    g = Grid.for_scene(scene)
    g.build(pos)
    off, ids = g.query_radius(scene.r, method=method)      # sizes tables, scratch and the id buffer
    g.sync()
    ids = torch.empty(int(off[-1]) * 2, dtype=torch.int32, device="cuda")
    step = lambda: (g.build(pos), g.query_radius(scene.r, method=method, out_offsets=off, out_ids=ids,
                                                  sync_total=False))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for k in range(2):
        off.zero_()
        graph.replay()
        torch.cuda.synchronize()
        g.sync()
        o = off.cpu().numpy()
        assert_csr_equal(o, ids[: o[-1]].cpu().numpy(), *oracle_radius(scene))
        # move the points in place (a small cyclic shift): the replay rebins them
        shifted = np.mod(scene.pos[:, :3] + np.float32(0.25 / 32), np.float32(1.0)).astype(np.float32)
        shifted = np.where(shifted >= 1.0, np.float32(0.0), shifted)
        scene.pos[:, :3] = shifted
        pos.copy_(torch.from_numpy(scene.pos))

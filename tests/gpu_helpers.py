"""Helpers for the parity tests: run a scene through the CUDA library and the
same seeded scene through the oracle, and compare."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_cs_0608108_b300 import Grid, synth


def to_dev(pos: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(pos, dtype=np.float32)).cuda()


def gpu_grid(scene: synth.Scene, r_max=None, capacity=None) -> Grid:
    g = Grid(scene.origin, scene.cell_size, scene.log2_cells, scene.cyclic_mask,
             scene.r if r_max is None else r_max, scene.n if capacity is None else capacity)
    return g.build(to_dev(scene.pos))


def gpu_radius(scene, r=None, method="sphere", include_self=False, sort=True, grid=None,
               walk="classes"):
    g = grid or gpu_grid(scene)
    off, ids = g.query_radius(scene.r if r is None else r, include_self=include_self,
                              method=method, sort=sort, walk=walk)
    g.sync()
    return off.cpu().numpy(), ids.cpu().numpy()


def oracle_radius(scene, r=None, queries=None, include_self=False):
    r = float(np.float32(scene.r if r is None else r))   # the radius the library receives
    q = np.arange(scene.n) if queries is None else np.asarray(queries)
    self_idx = None if include_self else q
    return oracle.radius(scene.pos, scene.pos[q], scene.box, scene.cyclic_mask, r, self_idx,
                         threads=0)


def assert_csr_equal(off_g, ids_g, off_o, ids_o):
    assert off_g.shape == off_o.shape
    bad = np.nonzero(off_g != off_o)[0]
    assert bad.size == 0, f"offsets differ first at query {bad[:5]}"
    assert np.array_equal(ids_g, ids_o), "neighbor ids differ"


def assert_sampled_equal(off_g, ids_g, scene, queries, r=None, include_self=False):
    off_o, ids_o = oracle_radius(scene, r, queries, include_self)
    for t, q in enumerate(queries):
        got = ids_g[off_g[q]:off_g[q + 1]]
        want = ids_o[off_o[t]:off_o[t + 1]]
        assert np.array_equal(got, want), f"query {q}: {len(got)} vs {len(want)} ids"

"""Parity of the fused neighbor reduction (energy and hand-written adjoint)
with the FP64 oracle: energy relative error and gradient global relative L2
error below 1e-4; the autograd path against FP64 central differences."""
import numpy as np
import pytest
import torch

import oracle
from paper_cs_0608108_b300 import Grid, neighbor_energy, synth

from gpu_helpers import gpu_grid, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-4


def gpu_reduce(scene, grad=True):
    g = gpu_grid(scene)
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    gr = torch.empty((scene.n, 4), dtype=torch.float32, device="cuda") if grad else None
    g.neighbor_reduce(scene.r, energy=e, grad=gr)
    g.sync()
    return float(e.item()), (gr.cpu().numpy()[:, :3] if grad else None), g


@pytest.mark.parametrize("mask", [7, 0, 5])
def test_energy_and_gradient_exact_small(mask):
    pos = synth.uniform_points(20_000, 60 + mask)
    if not mask & 2:
        pos[:10, 1] = np.float32(-0.2)     # outside points take part too
    scene = synth.Scene(pos, (0, 0, 0), 1 / 32, (5, 5, 5), mask, 1.5 / 32)
    E, G, _ = gpu_reduce(scene)
    e, g = oracle.reduce(scene.pos, np.arange(scene.n), scene.box, mask, scene.r)
    assert abs(E - e.sum()) <= TOL * e.sum()
    assert np.linalg.norm(G - g) <= TOL * np.linalg.norm(g)


def test_full_size_1m_energy_and_gradient_exact():
    # config 5 positions (1M uniform, 128^3 cyclic, r = 1.5 cells) and three
    # random-walk steps with rebinning: E and every gradient against the FP64
    # oracle through its bin lattice (all points, not a sample)
    scene = synth.uniform_1m_scene()
    g = Grid(scene.origin, scene.cell_size, scene.log2_cells, 7, scene.r, scene.n)
    pos = scene.pos
    for step in range(4):
        if step:
            pos = synth.random_walk_step(pos, synth.SEEDS["walk_1m"], step, 0.1 * scene.cell_size)
        g.build(to_dev(pos))
        e = torch.empty(1, dtype=torch.float64, device="cuda")
        gr = torch.empty((scene.n, 4), dtype=torch.float32, device="cuda")
        g.neighbor_reduce(scene.r, energy=e, grad=gr)
        g.sync()
        eo, go = oracle.reduce_all(pos, scene.box, 7, scene.r)
        G = gr.cpu().numpy()[:, :3]
        assert abs(float(e.item()) - eo.sum()) <= TOL * eo.sum()
        assert np.linalg.norm(G - go) <= TOL * np.linalg.norm(go)
        rms = np.sqrt((go ** 2).sum(axis=1).mean())
        assert np.abs(G - go).max() <= 1e-3 * rms


def test_full_size_1m_gradient_sampled():
    scene = synth.uniform_1m_scene()
    E, G, _ = gpu_reduce(scene)
    idx = np.random.default_rng(3).choice(scene.n, 2000, replace=False)
    e, g = oracle.reduce(scene.pos, idx, scene.box, 7, scene.r)
    assert np.linalg.norm(G[idx] - g) <= TOL * np.linalg.norm(g)
    # per-point error normalised by the RMS gradient
    rms = np.sqrt((g ** 2).sum(axis=1).mean())
    assert np.abs(G[idx] - g).max() <= 1e-3 * rms
    # E estimated from the sample (mean energy per point)
    assert abs(E / scene.n - e.mean()) <= 0.05 * e.mean()
    assert abs(G.sum(axis=0)).max() <= 1e-3 * np.abs(G).sum(axis=0).max()


def test_autograd_matches_oracle_and_finite_differences():
    pos_np = synth.uniform_points(3000, 12)
    scene = synth.Scene(pos_np, (0, 0, 0), 1 / 16, (4, 4, 4), 7, 0.09)
    g = Grid(scene.origin, scene.cell_size, scene.log2_cells, 7, scene.r, scene.n)
    x = to_dev(pos_np).requires_grad_(True)
    E = neighbor_energy(x, g, scene.r)
    (2.5 * E).backward()
    G = x.grad.cpu().numpy()[:, :3]
    e, go = oracle.reduce(pos_np, np.arange(scene.n), scene.box, 7, scene.r)
    assert abs(E.item() - e.sum()) <= TOL * e.sum()
    assert np.linalg.norm(G - 2.5 * go) <= TOL * np.linalg.norm(2.5 * go)
    assert np.all(x.grad.cpu().numpy()[:, 3] == 0)
    # FP64 central differences of the oracle energy on a subset
    h = 2.0 ** -16
    for i in range(0, 3000, 301):
        for a in range(3):
            p1, p0 = pos_np.copy(), pos_np.copy()
            p1[i, a] += np.float32(h)
            p0[i, a] -= np.float32(h)
            e1, _ = oracle.reduce(p1, np.arange(scene.n), scene.box, 7, scene.r)
            e0, _ = oracle.reduce(p0, np.arange(scene.n), scene.box, 7, scene.r)
            fd = (e1.sum() - e0.sum()) / (2 * h)
            assert abs(2.5 * fd - G[i, a]) <= 1e-3 * max(1.0, abs(G[i, a]))


def test_random_walk_steps_rebin_and_stay_exact():
    scene = synth.uniform_1m_scene(200_000)
    s = scene.cell_size
    g = Grid(scene.origin, s, scene.log2_cells, 7, scene.r, scene.n)
    pos = scene.pos
    for step in range(3):
        pos = synth.random_walk_step(pos, 99, step, 0.1 * s)
        g.build(to_dev(pos))
        e = torch.empty(1, dtype=torch.float64, device="cuda")
        gr = torch.empty((scene.n, 4), dtype=torch.float32, device="cuda")
        g.neighbor_reduce(scene.r, energy=e, grad=gr)
        g.sync()
        idx = np.arange(step, scene.n, 997)
        eo, go = oracle.reduce(pos, idx, scene.box, 7, scene.r)
        G = gr.cpu().numpy()[idx, :3]
        assert np.linalg.norm(G - go) <= TOL * np.linalg.norm(go)

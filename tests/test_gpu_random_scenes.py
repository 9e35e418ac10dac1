"""Seeded random scenes across the parameter space, every result against the
oracle: lattices of different shapes (anisotropic powers of two, cell sides
that are not powers of two, offset origins), every cyclic mask, uniform and
clustered points (some outside the region on non-cyclic axes), radii from
below a cell to several cells, all-agents radius lists through every method,
K-nearest queries (K from 1 to 64, ids, counts and distances), both
queries from random centers, the scenes as one batch, and the fused
reduction (energy and gradient within 1e-4 of FP64)."""
import numpy as np
import pytest

import oracle
from paper_cs_0608108_b300 import synth

from gpu_helpers import assert_csr_equal, gpu_grid, oracle_radius

pytestmark = pytest.mark.gpu


def random_scene(seed):
    rng = np.random.default_rng(seed)
    log2 = tuple(int(x) for x in rng.integers(3, 7, 3))
    s = float(np.float32(rng.choice([1 / 16, 1 / 32, 0.37, 0.0625 * 1.3])))
    origin = tuple(float(np.float32(x)) for x in rng.uniform(-2, 2, 3))
    mask = int(rng.integers(0, 8))
    box = tuple(s * (1 << w) for w in log2)
    n = int(rng.integers(500, 12_000))
    if rng.random() < 0.5:
        pos = synth.uniform_points(n, seed, box=box, origin=origin)
    else:   # clusters: crowded cells next to empty ones
        k = int(rng.integers(2, 9))
        c = rng.uniform(0, 1, (k, 3)) * np.array(box) + np.array(origin)
        lab = rng.integers(0, k, n)
        x = c[lab] + rng.normal(0, 0.6 * s, (n, 3))
        for a in range(3):
            if (mask >> a) & 1:   # wrapped into the box on cyclic axes
                x[:, a] = origin[a] + np.mod(x[:, a] - origin[a], box[a])
        pos = np.zeros((n, 4), np.float32)
        pos[:, :3] = x.astype(np.float32)
        for a in range(3):   # float32 rounding may land on the upper edge
            if (mask >> a) & 1:
                hi = np.float32(origin[a] + box[a])
                pos[:, a] = np.where(pos[:, a] >= hi, np.float32(origin[a]), pos[:, a])
    for a in range(3):   # a few points outside the region on non-cyclic axes
        if not (mask >> a) & 1:
            pos[a * 3:(a + 1) * 3, a] = np.float32(origin[a] - 0.5 * s if a % 2 else origin[a] + box[a] + 0.3 * s)
    # radius: below a cell to several cells, within what a cyclic axis allows
    gmin = min((1 << log2[a]) for a in range(3) if (mask >> a) & 1) if mask else 64
    rmax_cells = max(0.3, min(3.5, (gmin - 1) / 2 - 1.01))
    r = float(rng.uniform(0.3, rmax_cells)) * s
    return synth.Scene(pos, origin, s, log2, mask, r), rng


@pytest.mark.parametrize("seed", range(12))
def test_random_scene_radius_every_method(seed):
    scene, _ = random_scene(1000 + seed)
    off_o, ids_o = oracle_radius(scene)
    g = gpu_grid(scene)
    for method, walk in (("sphere", "classes"), ("sphere", "paper"), ("cube", "classes"), ("list", "classes"),
                         ("sphere_only", "planes")):
        off, ids = g.query_radius(scene.r, method=method, walk=walk)
        g.sync()
        assert_csr_equal(off.cpu().numpy(), ids.cpu().numpy(), off_o, ids_o)


@pytest.mark.parametrize("seed", range(12))
def test_random_scene_knn(seed):
    scene, rng = random_scene(2000 + seed)
    g = gpu_grid(scene)
    r = float(np.float32(scene.r))
    for k in sorted({int(rng.integers(1, 17)), int(rng.integers(17, 65))}):
        ids, d2, cnt = g.query_knn(k, r_max=scene.r)
        g.sync()
        oi, od, oc = oracle.knn(scene.pos, scene.pos, scene.box, scene.cyclic_mask, k, r, np.arange(scene.n))
        assert np.array_equal(cnt.cpu().numpy(), oc)
        assert np.array_equal(ids.cpu().numpy(), oi)
        fin = np.isfinite(od)
        assert np.array_equal(d2.cpu().numpy()[fin], od[fin].astype(np.float32))


@pytest.mark.parametrize("seed", range(8))
def test_random_scene_from_centers(seed):
    # caller-given centers: uniform over the region and a little beyond it on
    # non-cyclic axes, radius lists and K nearest against the oracle
    scene, rng = random_scene(3000 + seed)
    g = gpu_grid(scene)
    m = int(rng.integers(100, 4000))
    c = np.zeros((m, 4), np.float32)
    for a in range(3):
        lo, L = scene.origin[a], scene.box[a]
        if (scene.cyclic_mask >> a) & 1:
            x = (lo + rng.random(m) * L).astype(np.float32)
            x = np.where(x >= np.float32(lo + L), np.float32(lo), x)
        else:
            x = (lo - 0.1 * L + rng.random(m) * 1.2 * L).astype(np.float32)
        c[:, a] = x
    import torch
    cd = torch.from_numpy(c).cuda()
    off, ids = g.query_radius(scene.r, centers=cd)
    g.sync()
    r = float(np.float32(scene.r))
    off_o, ids_o = oracle.radius(scene.pos, c, scene.box, scene.cyclic_mask, r, None)
    assert_csr_equal(off.cpu().numpy(), ids.cpu().numpy(), off_o, ids_o)
    k = int(rng.integers(1, 65))
    ki, kd, kc = g.query_knn(k, r_max=scene.r, centers=cd)
    g.sync()
    oi, od, oc = oracle.knn(scene.pos, c, scene.box, scene.cyclic_mask, k, r, None)
    assert np.array_equal(kc.cpu().numpy(), oc) and np.array_equal(ki.cpu().numpy(), oi)
    fin = np.isfinite(od)
    assert np.array_equal(kd.cpu().numpy()[fin], od[fin].astype(np.float32))


@pytest.mark.parametrize("seed", range(3))
def test_random_scenes_in_one_batch(seed):
    # the random scenes above (uniform and clustered, every mask) served as
    # one batch under random planner choices, graph replays included
    import torch
    from paper_cs_0608108_b300 import Batch, default_batch_params
    from gpu_helpers import to_dev
    rng = np.random.default_rng(4000 + seed)
    scenes = [random_scene(5000 + 20 * seed + i)[0] for i in range(int(rng.integers(4, 20)))]
    ref = [oracle_radius(sc) for sc in scenes]
    p = default_batch_params()
    p["heavy_hits"] = float(rng.choice([0.0, 4.0, 24.0, 1e9]))
    p["q_tile"] = int(rng.choice([64, 128, 256]))
    p["branches"] = int(rng.integers(1, 9))
    p["blocks_per_sm"] = 2048 // p["q_tile"] // 2
    pos = [to_dev(sc.pos) for sc in scenes]
    offs = [torch.empty(sc.n + 1, dtype=torch.int64, device="cuda") for sc in scenes]
    ids = [torch.empty(int(o[-1]) + 1, dtype=torch.int32, device="cuda") for o, _ in ref]
    b = Batch(list(zip(scenes, pos)), offs, ids, params=p)
    for use_graph in (False, True, True):
        for t in ids:
            t.fill_(-7)
        b.run(use_graph=use_graph)
        totals = b.sync()
        for k, (off_o, ids_o) in enumerate(ref):
            o = offs[k].cpu().numpy()
            assert totals[k] == off_o[-1]
            assert_csr_equal(o, ids[k].cpu().numpy()[: o[-1]], off_o, ids_o)


@pytest.mark.parametrize("seed", range(6))
def test_random_scene_reduction(seed):
    # the fused reduction on the random scenes: energy and gradient within
    # 1e-4 of the FP64 oracle (global relative errors)
    import torch
    scene, _ = random_scene(6000 + seed)
    g = gpu_grid(scene)
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    gr = torch.empty((scene.n, 4), dtype=torch.float32, device="cuda")
    g.neighbor_reduce(scene.r, energy=e, grad=gr)
    g.sync()
    eo, go = oracle.reduce(scene.pos, np.arange(scene.n), scene.box, scene.cyclic_mask, float(np.float32(scene.r)))
    assert abs(float(e.item()) - eo.sum()) <= 1e-4 * max(eo.sum(), 1e-30)
    G = gr.cpu().numpy()[:, :3]
    assert np.linalg.norm(G - go) <= 1e-4 * max(np.linalg.norm(go), 1e-30)

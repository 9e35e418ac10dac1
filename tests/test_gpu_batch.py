"""Parity of the batched path (short-list scenes in one fused set of launches,
long-list scenes through their own pipelines, optionally replayed from a CUDA
graph) with the FP64 oracle and the single-scene path, scene by scene."""
import numpy as np
import pytest
import torch

from paper_cs_0608108_b300 import Batch, _native, synth

from gpu_helpers import assert_csr_equal, gpu_radius, oracle_radius, to_dev

pytestmark = pytest.mark.gpu


def make_batch(scenes, caps=None):
    pos = [to_dev(s.pos) for s in scenes]
    offs = [torch.empty(s.n + 1, dtype=torch.int64, device="cuda") for s in scenes]
    ids = [torch.empty(max(int(c), 1), dtype=torch.int32, device="cuda")
           for c in (caps or [64 * s.n + 64 for s in scenes])]
    return Batch(list(zip(scenes, pos)), offs, ids), offs, ids


def test_small_uneven_batch_matches_oracle_and_graph_replays():
    scenes = synth.batched_scenes(24, seed=123, n_lo=10, n_hi=20_000)
    scenes[3].pos = scenes[3].pos[:0]          # an empty scene
    ref = [oracle_radius(sc) for sc in scenes]
    b, offs, ids = make_batch(scenes, caps=[int(o[-1]) + 1 for o, _ in ref])
    b.run(use_graph=False)
    totals = b.sync()
    for k, sc in enumerate(scenes):
        off_o, ids_o = ref[k]
        o = offs[k].cpu().numpy()
        assert totals[k] == off_o[-1]
        assert_csr_equal(o, ids[k].cpu().numpy()[: o[-1]], off_o, ids_o)
    for _ in range(2):
        for t in ids:
            t.fill_(-7)
        b.run(use_graph=True)
        b.sync()
        for k, (off_o, ids_o) in enumerate(ref):
            o = offs[k].cpu().numpy()
            assert_csr_equal(o, ids[k].cpu().numpy()[: o[-1]], off_o, ids_o)


def test_batch_equals_looped_plain_path_on_seeded_scenes():
    scenes = synth.batched_scenes(16, seed=7, n_lo=1000, n_hi=60_000)
    plain = [gpu_radius(sc) for sc in scenes]
    b, offs, ids = make_batch(scenes, caps=[int(o[-1]) + 1 for o, _ in plain])
    b.run(use_graph=True)
    b.sync()
    for k, sc in enumerate(scenes):
        off_p, ids_p = plain[k]
        o = offs[k].cpu().numpy()
        assert np.array_equal(o, off_p)
        assert np.array_equal(ids[k].cpu().numpy()[: o[-1]], ids_p)


def test_batch_capacity_overflow_is_reported():
    scenes = synth.batched_scenes(4, seed=9, n_lo=2000, n_hi=3000)
    big = [int(oracle_radius(sc)[0][-1]) + 1 for sc in scenes]
    b, offs, ids = make_batch(scenes, caps=[1] + big[1:])
    b.run()
    with pytest.raises(_native.SIError) as ei:
        b.sync()
    assert ei.value.status == _native.SI_ERR_CAPACITY


@pytest.mark.parametrize("kind", ["long_lists_only", "short_lists_only"])
def test_batch_with_a_single_kind_of_scene(kind):
    # long lists: every scene runs its own pipeline on a graph branch, the
    # fused launches have nothing to do; short lists: the reverse
    if kind == "long_lists_only":
        scenes = [synth.Scene(synth.uniform_points(30_000, 61 + k), (0, 0, 0), 1 / 16, (4, 4, 4), 7 - k,
                              2.0 / 16) for k in range(3)]
    else:
        scenes = [synth.Scene(synth.uniform_points(5_000, 71 + k), (0, 0, 0), 1 / 32, (5, 5, 5), k,
                              1.0 / 32) for k in range(3)]
    plain = [gpu_radius(sc) for sc in scenes]
    b, offs, ids = make_batch(scenes, caps=[int(o[-1]) + 1 for o, _ in plain])
    for _ in range(3):
        for t in ids:
            t.fill_(-7)
        b.run(use_graph=True)
        totals = b.sync()
        for k, sc in enumerate(scenes):
            off_p, ids_p = plain[k]
            o = offs[k].cpu().numpy()
            assert totals[k] == off_p[-1]
            assert np.array_equal(o, off_p)
            assert np.array_equal(ids[k].cpu().numpy()[: o[-1]], ids_p)


def test_full_size_256_scene_batch_sampled():
    # the batched configuration at full size (256 scenes, 1,000-200,000
    # points each, lattices 16^3-128^3, r 1-3 cells, random cyclic masks),
    # replayed from its graph: every scene's total against the single-scene
    # path, and a sample of queries in every scene, element by element,
    # against the FP64 oracle
    from paper_cs_0608108_b300 import Grid
    scenes = synth.batched_scenes()
    totals = []
    for sc in scenes:
        g = Grid.for_scene(sc)
        g.build(to_dev(sc.pos))
        off, _ = g.query_radius(sc.r)
        totals.append(int(off[-1].item()))
        g.close()
    b, offs, ids = make_batch(scenes, caps=[t + 1 for t in totals])
    b.run(use_graph=False)
    b.sync()
    for _ in range(2):
        b.run(use_graph=True)
    got = b.sync()
    assert got == totals
    rng = np.random.default_rng(256)
    for k, sc in enumerate(scenes):
        if sc.n == 0:
            continue
        q = rng.choice(sc.n, min(6, sc.n), replace=False)
        off_o, ids_o = oracle_radius(sc, queries=q)
        o = offs[k].cpu().numpy()
        lst = ids[k].cpu().numpy()
        assert o[-1] == totals[k]
        for t, qi in enumerate(q):
            assert np.array_equal(lst[o[qi]:o[qi + 1]], ids_o[off_o[t]:off_o[t + 1]]), (k, qi)


def test_tuned_batch_matches_oracle_and_caches(tmp_path):
    # the planner's choices timed on the GPU (a few candidates, including
    # every scene fused and every scene on its own pipeline), the fastest
    # kept in a cache file; the tuned batch's lists are the oracle's
    import os
    from paper_cs_0608108_b300 import tune_batch
    scenes = synth.batched_scenes(12, seed=321, n_lo=500, n_hi=30_000)
    ref = [oracle_radius(sc) for sc in scenes]
    pos = [to_dev(s.pos) for s in scenes]
    offs = [torch.empty(s.n + 1, dtype=torch.int64, device="cuda") for s in scenes]
    ids = [torch.empty(int(o[-1]) + 1, dtype=torch.int32, device="cuda") for o, _ in ref]
    cands = [{"heavy_hits": h, "q_tile": t, "branches": 4, "blocks_per_sm": 4}
             for h, t in ((0.0, 128), (24.0, 64), (24.0, 256), (1e9, 128))]
    cache = os.path.join(tmp_path, "tune.json")
    params, info = tune_batch(list(zip(scenes, pos)), offs, ids, cache=cache, candidates=cands, reps=2)
    assert not info["cached"] and len(info["ms"]) == 4 and params in cands
    again, info2 = tune_batch(list(zip(scenes, pos)), offs, ids, cache=cache, candidates=cands)
    assert info2["cached"] and again == params
    for cand in (params, cands[0], cands[3]):
        b = Batch(list(zip(scenes, pos)), offs, ids, params=cand)
        for t in ids:
            t.fill_(-7)
        b.run(use_graph=True)
        b.run(use_graph=True)
        b.sync()
        for k, (off_o, ids_o) in enumerate(ref):
            o = offs[k].cpu().numpy()
            assert_csr_equal(o, ids[k].cpu().numpy()[: o[-1]], off_o, ids_o)
        b.close()

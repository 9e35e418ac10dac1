"""Host logic of the batch planner's tuning cache (CPU only): the cache key
of a batch depends on each scene's point-count bucket, lattice, radius in
cells, load bucket and cyclic mask, not on the order of the scenes; a cached
entry is returned without timing anything."""
import json
import os

import numpy as np

from paper_cs_0608108_b300 import batch_scene_key, batch_signature, synth, tune_batch


def scene(n, w=5, d=1.5, mask=7, seed=1):
    s = 1.0 / (1 << w)
    return synth.Scene(synth.uniform_points(n, seed), (0, 0, 0), s, (w, w, w), mask, d * s)


def test_signature_ignores_order_and_follows_each_key_part():
    base = [scene(1000), scene(5000, w=6), scene(20000, d=2.5, mask=3)]
    sig = batch_signature(base)
    assert batch_signature(base[::-1]) == sig
    assert batch_signature([base[1], base[2], base[0]]) == sig
    # inside a bucket: same key (1000 vs 1100 points round to the same log2)
    assert batch_scene_key(scene(1100)) == batch_scene_key(scene(1000))
    variants = [
        [scene(4000)] + base[1:],                    # point-count bucket
        [scene(1000, w=4)] + base[1:],               # lattice (and load)
        [scene(1000, d=2.0)] + base[1:],             # radius in cells
        [scene(1000, mask=5)] + base[1:],            # cyclic mask
    ]
    sigs = {batch_signature(v) for v in variants}
    assert sig not in sigs and len(sigs) == len(variants)
    assert batch_signature(base, flags=2) != sig
    k = batch_scene_key(scene(1000, w=5, d=1.5))
    assert k[0] == 10 and k[1] == (5, 5, 5) and k[2] == 1.5 and k[4] == 7
    assert k[3] == int(round(2 * np.log2(1000 / 32 ** 3)))


def test_cached_entry_is_returned_without_timing(tmp_path):
    scenes = [scene(2000, seed=3), scene(3000, seed=4)]
    sig = batch_signature(scenes)
    cache = os.path.join(tmp_path, "tune.json")
    want = {"heavy_hits": 64.0, "q_tile": 256, "branches": 4, "blocks_per_sm": 4}
    with open(cache, "w") as fh:
        json.dump({sig: {"params": want, "ms": 1.0, "scenes": 2}}, fh)
    # no device tensors are touched on a hit: the pairs carry None positions
    params, info = tune_batch([(s, None) for s in scenes], None, None, cache=cache)
    assert params == want and info["cached"] and info["signature"] == sig

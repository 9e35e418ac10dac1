"""The algorithmic pair count behind the bench's ALU roofline: the points of
every cell that meets each query's sphere (exact per-query culling), checked
against a direct enumeration of the cells on small scenes.  CPU only."""
import itertools

import numpy as np
import pytest

import bench
from paper_cs_0608108_b300 import synth


def cell_start(scene):
    w = np.array(scene.log2_cells)
    G = 1 << w
    u = (scene.pos[:, :3].astype(np.float64) - np.array(scene.origin)) / scene.cell_size
    c = np.clip(np.floor(u).astype(np.int64), 0, G - 1)
    key = (c[:, 2] << (w[0] + w[1])) | (c[:, 1] << w[0]) | c[:, 0]
    cnt = np.bincount(key, minlength=(1 << int(w.sum())) + 1)
    return np.concatenate([[0], np.cumsum(cnt)])


def direct(scene, start):
    """Every cell of the lattice and of its 26 cyclic images (when cyclic),
    tested against each query by its box distance."""
    w = scene.log2_cells
    G = 1 << w[0]
    d = scene.r / scene.cell_size
    cnt = np.diff(start)
    lo, hi = (-G, 2 * G) if scene.cyclic_mask == 7 else (0, G)
    t = np.array(list(itertools.product(range(lo, hi), repeat=3)))   # (z, y, x) image cells
    t = t[:, ::-1]                                                     # as (x, y, z)
    tw = t % G
    key = (tw[:, 2] << (w[0] + w[1])) | (tw[:, 1] << w[0]) | tw[:, 0]
    tot = 0
    for qp in scene.pos[:, :3].astype(np.float64) / scene.cell_size:
        c = np.minimum(np.floor(qp).astype(int), G - 1)
        f = qp - c
        o = t - c
        gap = np.where(o > 0, o - f, np.where(o < 0, f - o - 1, 0.0))
        tot += cnt[key[(gap ** 2).sum(axis=1) <= d * d]].sum()
    return tot


@pytest.mark.parametrize("mask", [7, 0])
def test_candidate_pairs_match_direct_enumeration(mask):
    scene = synth.Scene(synth.uniform_points(400, 5 + mask), (0, 0, 0), 1 / 8, (3, 3, 3), mask, 1.7 / 8)
    start = cell_start(scene)
    cls = np.zeros(len(start) - 1, dtype=np.int64)
    got = bench.candidate_pairs(scene, start, cls, sample=10 ** 9)
    assert got[0] == direct(scene, start)
    assert got[1] == got[2] == got[3] == 0


def test_candidate_pairs_split_by_class_and_scaled_sample():
    scene = synth.Scene(synth.gaussian_mixture_points(40_000, 3, n_comp=4, sigma=0.03), (0, 0, 0), 1 / 16,
                        (4, 4, 4), 7, 1.5 / 16)
    start = cell_start(scene)
    cls = bench.cell_classes(start, scene.log2_cells)
    full = bench.candidate_pairs(scene, start, cls, sample=10 ** 9)
    half = bench.candidate_pairs(scene, start, cls, sample=scene.n // 4)
    assert sum(full.values()) > 0 and full[1] + full[3] > 0
    # a quarter sample scaled up estimates the total within a few percent
    assert abs(sum(half.values()) - sum(full.values())) < 0.05 * sum(full.values())


def test_cell_classes_follow_the_binning_rule():
    """Heavy: >= 8 points, or >= 3 with >= 12 in the cell and its two packed
    neighbours; large heavy: heavy with >= 768 in the 27 cells around it (y, z
    wrapped, x clipped); dense: not heavy, >= 24 around it; the outside cell
    dense with >= 24 points."""
    scene = synth.Scene(synth.gaussian_mixture_points(30_000, 9, n_comp=6, sigma=0.02), (0, 0, 0), 1 / 16,
                        (4, 4, 4), 7, 1.5 / 16)
    start = cell_start(scene)
    cls = bench.cell_classes(start, scene.log2_cells)
    cnt = np.diff(start)
    G = 16
    nc = G ** 3
    for key in range(nc):
        x, y, z = key % G, (key // G) % G, key // (G * G)
        row = start[min(key + 2, nc)] - start[max(key - 1, 0)] if 1 <= key <= nc - 2 else 0
        heavy = cnt[key] >= 8 or (cnt[key] >= 3 and row >= 12)
        n27 = 0
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    xx = x + dx
                    if 0 <= xx < G:
                        n27 += cnt[((z + dz) % G) * G * G + ((y + dy) % G) * G + xx]
        want = (3 if n27 >= 768 else 1) if heavy else (2 if n27 >= 24 else 0)
        assert cls[key] == want, key
    assert cls[nc] == (2 if cnt[nc] >= 24 else 0)


def test_grouped_cells_rule():
    # the group split the bench predicts, against a per-cell reading of the
    # rule: a non-empty heavy cell (small class) of at most 128 points is
    # grouped when its aligned 2x2x2 block holds another such cell
    pos = synth.gaussian_mixture_points(30_000, 5, n_comp=6, sigma=0.08)
    scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), 7, 1.5 / 16)
    start = cell_start(scene)
    cls = bench.cell_classes(start, scene.log2_cells)
    got = bench.grouped_cells(cls, start, scene.log2_cells, 1.5)
    cnt = np.diff(start)
    G = 16
    want = np.zeros_like(got)
    for c in range(G ** 3):
        if cls[c] != 1 or cnt[c] == 0 or cnt[c] > 128:
            continue
        x, y, z = c % G, (c // G) % G, c // (G * G)
        mates = 0
        for k, j, i in itertools.product(range(2), repeat=3):
            c2 = (x & ~1) + i + G * ((y & ~1) + j) + G * G * ((z & ~1) + k)
            mates += cls[c2] == 1 and cnt[c2] > 0
        want[c] = mates >= 2
    assert np.array_equal(got, want) and want.sum() > 20 and (cls == 1).sum() > want.sum()
    # too small a lattice for the group rows at this distance: nothing grouped
    assert not bench.grouped_cells(cls, start, scene.log2_cells, 7.2).any()

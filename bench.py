"""Benchmark of the spherical-index neighborhood queries on B300.

Default (N=1): the all-agents fixed-radius query at 1M points on a 128^3
fully cyclic lattice, r = 1.5 cell sides, with both seeded distributions
(uniform and 64-component Gaussian mixture).  One step = one pass of the hot
path over both point clouds: bin (key, histogram, scan, scatter) and query
(count, scan, write, per-list id sort).  Other workloads: --workload
knn_4m | batched | walk_1m | tiny | radius_1m_cube.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle (FP64
brute force) on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "all-agent radius queries/s and HBM-roofline % at 1M pts, batched/fused vs plain, exact sets"
L2_BYTES = 126 * 2 ** 20


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def src_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_cs_0608108_b300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    from the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p):
        return None
    cur = src_hash()
    for line in open(p):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == kernel and f[1] == workload:
            return float(f[2]) if f[3] == cur else None
    return None


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.out = ""

    def summary(self):
        rows = []
        for line in (getattr(self, "out", "") or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 6:
                try:
                    rows.append((float(f[0]), float(f[1]), f[2:6]))
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons, "samples": len(rows)}


def dist_setup():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


# ---------------------------------------------------------------------------
# workloads (GPU arm)
# ---------------------------------------------------------------------------
def cell_classes(start, log2_cells):
    """Class of every cell as the binning assigns it: heavy 1 (>= 8 points,
    or >= 3 with >= 12 in the cell and its two x-neighbours), large heavy 3
    (heavy with >= 768 points in the 27 cells around it), dense 2 (not heavy,
    >= 24 points around it), light 0 (the rest); the last entry is the
    outside cell."""
    cnt = np.diff(start).astype(np.int64)
    nc = len(cnt) - 1                # lattice cells; key nc is the outside cell
    row = np.zeros(nc + 1, dtype=np.int64)
    if nc >= 3:
        key = np.arange(1, nc - 1)
        row[1:nc - 1] = start[key + 2] - start[key - 1]
    heavy = (cnt >= 8) | ((cnt >= 3) & (row >= 12))
    heavy[-1] = False
    wx, wy, wz = log2_cells
    c3 = cnt[:nc].reshape(1 << wz, 1 << wy, 1 << wx)
    xs = c3.copy()
    xs[:, :, 1:] += c3[:, :, :-1]
    xs[:, :, :-1] += c3[:, :, 1:]          # x clipped at the region's ends
    n27 = np.zeros_like(c3)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            n27 += np.roll(np.roll(xs, dz, 0), dy, 1)   # y, z wrapped
    n27 = np.append(n27.ravel(), cnt[nc])
    cls = np.where(heavy, np.where(n27 >= 768, 3, 1), np.where(n27 >= 24, 2, 0))
    cls[-1] = np.where(cnt[nc] >= 24, 2, 0)
    return cls


def grouped_cells(cls, start, log2_cells, d):
    """Heavy cells of the small class served by the 2x2x2 group kernel: the
    non-empty ones of at most 128 queries whose aligned group holds another
    non-empty heavy cell of that class (the library's k_group_list rule;
    groups whose candidates overflow a block at run time are not predicted),
    on lattices with at least 2 reach + 2 cells per axis."""
    cnt = np.diff(start).astype(np.int64)
    G = [1 << w for w in log2_cells]
    reach = int(np.floor(d)) + 1
    out = np.zeros(len(cls), dtype=bool)
    if min(log2_cells) < 1 or min(G) < 2 * reach + 2:
        return out
    nc = len(cnt) - 1
    hs = ((cls[:nc] == 1) & (cnt[:nc] > 0)).reshape(G[2], G[1], G[0])
    blk = hs.reshape(G[2] // 2, 2, G[1] // 2, 2, G[0] // 2, 2).sum(axis=(1, 3, 5))
    per = np.repeat(np.repeat(np.repeat(blk, 2, 0), 2, 1), 2, 2)
    out[:nc] = (hs & (per >= 2)).ravel() & (cnt[:nc] <= 128)
    return out


def candidate_pairs(scene, start, cls, sample=131_072):
    """Algorithmic pair tests of the spherical index, by query class: for
    each query point, the points of every cell that meets its sphere (exact
    per-query cell culling, cyclic wrap; cells leaving a non-cyclic region
    skipped), summed over a fixed sample of queries and scaled to all."""
    pos = scene.pos
    n = len(pos)
    if n == 0:
        return {c: 0.0 for c in range(5)}
    step = max(1, n // sample)
    q = pos[::step, :3].astype(np.float64)
    w = np.array(scene.log2_cells)
    G = 1 << w
    u = (q - np.array(scene.origin)) / scene.cell_size
    c = np.clip(np.floor(u).astype(np.int64), 0, G - 1)
    f = u - c
    d = scene.r / scene.cell_size
    D = int(np.ceil(d))
    cnt = np.diff(start).astype(np.int64)
    qcls = cls[(c[:, 2] << (w[0] + w[1])) | (c[:, 1] << w[0]) | c[:, 0]]
    tot = np.zeros(len(q))
    for oz in range(-D, D + 1):
        for oy in range(-D, D + 1):
            for ox in range(-D, D + 1):
                o = np.array([ox, oy, oz])
                gap = np.where(o > 0, o - f, np.where(o < 0, f - o - 1, 0.0))
                ok = (gap * gap).sum(axis=1) <= d * d
                t = c + o
                for a in range(3):
                    if (scene.cyclic_mask >> a) & 1:
                        t[:, a] %= G[a]
                    else:
                        ok &= (t[:, a] >= 0) & (t[:, a] < G[a])
                t = np.clip(t, 0, G - 1)
                key = (t[:, 2] << (w[0] + w[1])) | (t[:, 1] << w[0]) | t[:, 0]
                tot += np.where(ok, cnt[key], 0)
    return {k: float(tot[qcls == k].sum()) * step for k in range(5)}


class RadiusWork:
    """Bin + all-agents radius query for a list of scenes."""

    def __init__(self, scenes, method="sphere", walk="classes"):
        import torch
        from paper_cs_0608108_b300 import Grid
        self.scenes = scenes
        self.method = method
        self.walk = walk
        self.pos = [torch.from_numpy(s.pos).cuda() for s in scenes]
        self.grids = [Grid.for_scene(s) for s in scenes]
        self.off, self.ids, self.totals = [], [], []
        for g, p, s in zip(self.grids, self.pos, scenes):
            g.build(p)
            off, ids = g.query_radius(s.r, method=method, walk=walk)
            g.sync()
            self.totals.append(int(off[-1].item()))
            self.off.append(off)
            self.ids.append(torch.empty(max(self.totals[-1], 1), dtype=torch.int32, device="cuda"))
        self.queries = sum(s.n for s in scenes)
        # independent scenes run on streams of their own (forked from and
        # joined to the current stream, so graph capture follows them)
        self.streams = [torch.cuda.Stream() for _ in scenes] if len(scenes) > 1 else None
        self.serial = False                  # one stream (the per-kernel timing pass)

    def step(self):
        import torch
        cur = torch.cuda.current_stream()
        for k, (g, p, s, off, ids) in enumerate(zip(self.grids, self.pos, self.scenes, self.off, self.ids)):
            if self.streams is None or self.serial:
                g.build(p)
                g.query_radius(s.r, method=self.method, walk=self.walk, out_offsets=off, out_ids=ids,
                               sync_total=False)
                continue
            self.streams[k].wait_stream(cur)
            with torch.cuda.stream(self.streams[k]):
                g.build(p)
                g.query_radius(s.r, method=self.method, walk=self.walk, out_offsets=off, out_ids=ids,
                               sync_total=False)
        if self.streams is not None and not self.serial:
            for st in self.streams:
                cur.wait_stream(st)

    def check(self):
        for g in self.grids:
            g.sync()

    def cell_split(self, k):
        """Per kernel family, the (fraction of queries, fraction of hits) it
        serves in scene k, from the cell classes the binning assigns: heavy
        (>= 8 points, or >= 3 with >= 12 in the cell and its two x-neighbours),
        large heavy (>= 768 points in the 27 cells around it), dense (not
        heavy, >= 24 points around it), light (the rest).  Cells that overflow
        the small configuration at run time are counted as small."""
        start, _, perm = (t.cpu().numpy() for t in self.grids[k].cell_arrays())
        cnt = np.diff(start).astype(np.int64)
        cls = self.classes(k, start)
        slot_cls = np.repeat(cls, cnt.clip(min=0))[: len(perm)]
        off = self.off[k].cpu().numpy()
        lens = np.diff(off)
        tot = max(lens.sum(), 1)
        out = {}
        for name, c in (("light", 0), ("small", 1), ("dense", 2), ("large", 3), ("group", 4)):
            sel = slot_cls == c
            out[name] = (sel.mean() if len(perm) else 0.0, lens[perm[sel]].sum() / tot)
        return out

    def classes(self, k, start):
        """Cell classes of scene k as the binning assigns them, with the heavy
        cells served by the group kernel relabelled 4."""
        s = self.scenes[k]
        cls = cell_classes(start, s.log2_cells)
        if self.method == "cube":
            cls[:] = 0
            return cls
        cls = cls.copy()
        cls[grouped_cells(cls, start, s.log2_cells, s.r / s.cell_size)] = 4
        return cls

    def algorithmic_bytes(self):
        """Per-kernel minimum DRAM bytes of one launch, averaged over the scenes:
        each structure touched once by the queries that kernel serves."""
        out = {}
        for k, (s, tot) in enumerate(zip(self.scenes, self.totals)):
            n, C = s.n, (1 << sum(s.log2_cells)) + 1
            f = self.cell_split(k)
            fl, fd, fs, fb, fg = (f[c][0] for c in ("light", "dense", "small", "large", "group"))
            tl, td, ts, tb, tg = (f[c][1] for c in ("light", "dense", "small", "large", "group"))
            # per-query kernels: the query's point, index and list entry, the
            # cell starts, the count (count pass) or offset (write pass)
            q_b = 16 * n + 4 * n + 4 * n + 8 * n
            # cell kernels: the queries' points and indices, the cell starts,
            # the counts (the per-cell records in between are not algorithmic)
            c_b = 16 * n + 4 * n + 8 * n
            per = {
                "k_bin_key": 16 * n + 8 * n + 8 * C,
                "k_bin_scatter": 8 * n + 16 * n + 4 * C + 16 * n + 4 * n,
                "k_radius_count": fl * q_b + fl * 4 * C,
                "k_radius_write": fl * q_b + fl * 4 * C + tl * 4 * tot,
                "k_radius_dense_count": fd * q_b + fd * 4 * C,
                "k_radius_dense_write": fd * q_b + fd * 4 * C + td * 4 * tot,
                "k_cell": fs * c_b + fs * 4 * C,
                "k_cell_group": fg * c_b + fg * 4 * C,
                "k_cell_large": fb * c_b + fb * 4 * C,
                # the lists of the heavy queries, with their offsets and
                # indices: the warp-per-item expansion serves the small and
                # grouped cells, the block-per-cell one the large cells
                "k_expand_items": (fs + fg) * (4 * n + 8 * n) + (ts + tg) * 4 * tot,
                "k_cell_expand": fb * (4 * n + 8 * n) + tb * 4 * tot,
                "k_radius_count_cube": 16 * n + 4 * n + 4 * C + 8 * n,
                "k_radius_write_cube": 16 * n + 4 * n + 4 * C + 8 * n + 4 * tot,
                "k_radius_count_planes": 16 * n + 4 * n + 4 * C + 8 * n,
                "k_radius_write_planes": 16 * n + 4 * n + 4 * C + 8 * n + 4 * tot,
            }
            for kk, v in per.items():
                out.setdefault(kk, []).append(v)
        return {kk: float(np.mean(v)) for kk, v in out.items()}

    def step_bytes(self):
        tot = 0
        for s, t in zip(self.scenes, self.totals):
            n, C = s.n, (1 << sum(s.log2_cells)) + 1
            tot += (16 + 20) * n + 4 * C + (16 + 4) * n + 4 * C + 8 * n + 4 * t
        return tot

    def algorithmic_pairs(self):
        """Per pair-testing kernel, the algorithmic pair tests of one launch
        (candidate_pairs of the queries it serves), averaged over the scenes."""
        if self.method == "cube":
            return {}
        out = {}
        for k, s in enumerate(self.scenes):
            start, _, _ = (t.cpu().numpy() for t in self.grids[k].cell_arrays())
            p = candidate_pairs(s, start, self.classes(k, start))
            out.setdefault("k_radius_count_planes", []).append(sum(p.values()))
            out.setdefault("k_radius_write_planes", []).append(sum(p.values()))
            for name, c in (("k_radius_count", 0), ("k_radius_write", 0), ("k_radius_dense_count", 2),
                            ("k_radius_dense_write", 2), ("k_cell", 1), ("k_cell_large", 3),
                            ("k_cell_group", 4)):
                out.setdefault(name, []).append(p[c])
        return {kk: float(np.mean(v)) for kk, v in out.items()}

    def step_pairs(self):
        """Candidate pair tests of one step, every scene, every cell class."""
        if self.method == "cube":
            return None
        tot = 0
        for k, s in enumerate(self.scenes):
            start, _, _ = (t.cpu().numpy() for t in self.grids[k].cell_arrays())
            tot += sum(candidate_pairs(s, start, self.classes(k, start)).values())
        return float(tot)


def host_link():
    """Copy rate of the host link (page-locked host memory), each direction
    on its own: best of three 512 MiB copies, GB/s."""
    import torch
    n = 1 << 27
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    h = torch.empty(n, dtype=torch.int32).pin_memory()
    out = {}
    for name, dst, src in (("d2h_gbs", h, d), ("h2d_gbs", d, h)):
        best = 0.0
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            best = max(best, 4 * n / (time.perf_counter() - t0) / 1e9)
        out[name] = best
    del d, h
    return out


def e2e_radius_host(work, steps, warmup):
    """The metric end to end through the C ABI with host buffers
    (si_query_radius_host): every step hands each scene's points in
    page-locked host memory to the library, which copies them in, bins,
    queries and copies the CSR result back to page-locked host memory before
    returning; the scenes' calls are made from host threads of their own.
    Timed by the host clock around whole steps (the calls return only when
    their lists are in host memory)."""
    import torch
    hpos = [torch.from_numpy(s.pos).pin_memory() for s in work.scenes]
    hoff = [torch.empty(s.n + 1, dtype=torch.int64).pin_memory() for s in work.scenes]
    hids = [torch.empty(max(t, 1), dtype=torch.int32).pin_memory() for t in work.totals]

    # one host thread and stream per scene, as the device-side step runs
    # them (the call blocks its thread until the scene's lists are home)
    from concurrent.futures import ThreadPoolExecutor
    streams = [torch.cuda.Stream() for _ in work.scenes]
    pool = ThreadPoolExecutor(len(work.scenes))

    def scene(k):
        with torch.cuda.stream(streams[k]):
            if work.grids[k].query_radius_host(hpos[k], work.scenes[k].r, hoff[k], hids[k]) != work.totals[k]:
                raise RuntimeError("end-to-end total differs from the device path's")

    def one():
        for f in [pool.submit(scene, k) for k in range(len(work.scenes))]:
            f.result()
    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) * 1e3 / steps
    pool.shutdown()
    for k in range(len(work.scenes)):      # what reached the host equals the device path's result
        if not torch.equal(hoff[k], work.off[k].cpu()):
            raise RuntimeError("end-to-end offsets do not match the device result")
    ms = wall
    bi = sum(16 * s.n for s in work.scenes)
    bo = sum(8 * (s.n + 1) + 4 * t for s, t in zip(work.scenes, work.totals))
    return ms, wall, bi, bo


def e2e_radius(work, steps, warmup):
    """Same metric through the Python API with host buffers: every step copies
    the points in from pinned host memory, bins and queries, and copies the
    CSR result back to pinned host memory.  Steps are pipelined: a step's
    lists go out on a copy stream (into one of two device output sets) while
    the next step's points come in and are queried, so the host link, the
    bound here, stays busy; the timed region ends when the last copy lands."""
    import torch
    hpos = [torch.from_numpy(s.pos).pin_memory() for s in work.scenes]
    hoff = [torch.empty(s.n + 1, dtype=torch.int64).pin_memory() for s in work.scenes]
    hids = [torch.empty(max(t, 1), dtype=torch.int32).pin_memory() for t in work.totals]
    dpos = [torch.empty_like(p, device="cuda") for p in hpos]
    offs = [work.off, [o.clone() for o in work.off]]
    idss = [work.ids, [i.clone() for i in work.ids]]
    comp = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    done = [[None] * len(work.scenes) for _ in range(2)]

    def one(t):
        b = t % 2
        for k, (g, s) in enumerate(zip(work.grids, work.scenes)):
            dpos[k].copy_(hpos[k], non_blocking=True)
            g.build(dpos[k])
            if done[b][k] is not None:
                comp.wait_event(done[b][k])     # the output set's previous copy has landed
            g.query_radius(s.r, walk=work.walk, out_offsets=offs[b][k], out_ids=idss[b][k], sync_total=False)
            ready = torch.cuda.Event()
            ready.record(comp)
            copy.wait_event(ready)
            with torch.cuda.stream(copy):
                hoff[k].copy_(offs[b][k], non_blocking=True)
                hids[k][: work.totals[k]].copy_(idss[b][k][: work.totals[k]], non_blocking=True)
            landed = torch.cuda.Event()
            landed.record(copy)
            done[b][k] = landed
    for t in range(warmup):
        one(t)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(comp)
    for t in range(steps):
        one(warmup + t)
    comp.wait_stream(copy)
    b.record(comp)
    b.synchronize()
    for g in work.grids:
        g.sync()
    last = (warmup + steps - 1) % 2
    for k in range(len(work.scenes)):      # what reached the host is the last step's result
        if not torch.equal(hoff[k], offs[last][k].cpu()):
            raise RuntimeError("end-to-end copy does not match the device result")
    ms = a.elapsed_time(b) / steps
    bi = sum(16 * s.n for s in work.scenes)
    bo = sum(8 * (s.n + 1) + 4 * t for s, t in zip(work.scenes, work.totals))
    return ms, bi, bo


class CentersWork:
    """Bin + radius query from m caller-given centers (no self exclusion)."""

    def __init__(self, scene, centers):
        import torch
        from paper_cs_0608108_b300 import Grid
        self.scene = scene
        self.centers_np = centers
        self.pos = torch.from_numpy(scene.pos).cuda()
        self.centers = torch.from_numpy(centers).cuda()
        self.grid = Grid.for_scene(scene)
        self.grid.build(self.pos)
        off, _ = self.grid.query_radius(scene.r, centers=self.centers)
        self.grid.sync()
        self.total = int(off[-1].item())
        self.off = off
        self.ids = torch.empty(max(self.total, 1), dtype=torch.int32, device="cuda")
        self.queries = centers.shape[0]

    def step(self):
        self.grid.build(self.pos)
        self.grid.query_radius(self.scene.r, centers=self.centers, out_offsets=self.off, out_ids=self.ids,
                               sync_total=False)

    def check(self):
        self.grid.sync()

    def _split(self):
        """(fraction of centers, fraction of hits) served per thread (light
        cells) and per warp (the rest), from the cell classes of the centers'
        cells."""
        s = self.scene
        start, _, _ = (t.cpu().numpy() for t in self.grid.cell_arrays())
        cls = cell_classes(start, s.log2_cells)
        u = ((self.centers_np[:, :3] - np.array(s.origin, np.float32)) *
             np.float32(1.0 / s.cell_size)).astype(np.int64)
        w = s.log2_cells
        u = np.minimum(np.maximum(u, 0), [(1 << a) - 1 for a in w])
        key = (u[:, 2] << (w[0] + w[1])) | (u[:, 1] << w[0]) | u[:, 0]
        light = cls[key] == 0
        lens = np.diff(self.off.cpu().numpy())
        tot = max(lens.sum(), 1)
        return light.mean(), lens[light].sum() / tot

    def algorithmic_pairs(self):
        """The list method tests every (center, point) pair."""
        p = float(self.scene.n) * self.queries
        return {"k_radius_all_count": p, "k_radius_all_write": p}

    def algorithmic_bytes(self):
        s, m = self.scene, self.queries
        n, C = s.n, (1 << sum(s.log2_cells)) + 1
        fl, tl = self._split()
        q_b = 16 * m + 4 * m + 8 * m   # the center, its input index, its count or offset
        return {"k_bin_key": 16 * n + 8 * n + 8 * C,
                "k_bin_scatter": 8 * n + 16 * n + 4 * C + 16 * n + 4 * n,
                "k_center_key": 16 * m + 8 * m,
                "k_center_scatter": 16 * m + 8 * m + 16 * m + 4 * m + 4 * m,
                "k_radius_count": fl * q_b + 4 * C,
                "k_radius_write": fl * q_b + 4 * C + tl * 4 * self.total,
                "k_radius_dense_count": (1 - fl) * q_b + 4 * C,
                "k_radius_dense_write": (1 - fl) * q_b + 4 * C + (1 - tl) * 4 * self.total,
                # list method: the points once, each center, its count or offset, the lists
                "k_radius_all_count": 16 * n + 16 * m + 4 * m + 8 * m,
                "k_radius_all_write": 16 * n + 16 * m + 4 * m + 8 * m + 4 * self.total}

    def step_bytes(self):
        s, m = self.scene, self.queries
        n, C = s.n, (1 << sum(s.log2_cells)) + 1
        return 36 * n + 4 * C + 20 * n + 4 * C + 64 * m + 2 * 28 * m + 4 * C + 4 * self.total


class KnnWork:
    def __init__(self, scene, ks=(16, 64), method="sphere"):
        import torch
        from paper_cs_0608108_b300 import Grid
        self.scene = scene
        self.ks = ks
        self.pos = torch.from_numpy(scene.pos).cuda()
        self.grid = Grid.for_scene(scene)
        self.out = {k: (torch.empty((scene.n, k), dtype=torch.int32, device="cuda"),
                        torch.empty((scene.n, k), dtype=torch.float32, device="cuda"),
                        torch.empty(scene.n, dtype=torch.int32, device="cuda")) for k in ks}
        self.queries = scene.n * len(ks)
        self.method = method

    def step(self):
        self.grid.build(self.pos)
        for k in self.ks:
            self.grid.query_knn(k, r_max=self.scene.r, out=self.out[k], method=self.method)

    def check(self):
        self.grid.sync()

    def algorithmic_bytes(self):
        n, C = self.scene.n, (1 << sum(self.scene.log2_cells)) + 1
        kb = float(np.mean([16 * n + 4 * n + 4 * C + 8 * k * n + 4 * n for k in self.ks]))
        return {"k_knn_lane": kb, "k_knn_warp": kb, "k_knn": kb, "k_knn_cube": kb, "k_bin_key": 24 * n + 8 * C,
                "k_bin_scatter": 48 * n + 4 * C}

    def step_bytes(self):
        n, C = self.scene.n, (1 << sum(self.scene.log2_cells)) + 1
        return 36 * n + 4 * C + sum(20 * n + 4 * C + 8 * k * n + 4 * n for k in self.ks)


class WalkWork:
    """Random-walk timestep: rebin, energy kernel, adjoint kernel (autograd)."""

    def __init__(self, scene, n_pos=4):
        import torch
        from paper_cs_0608108_b300 import Grid
        self.scene = scene
        s = scene.cell_size
        pos = scene.pos
        self.frames = []
        for t in range(n_pos):
            pos = __import__("paper_cs_0608108_b300.synth", fromlist=["x"]).random_walk_step(
                pos, 0x5A1, t, 0.1 * s)
            self.frames.append(torch.from_numpy(pos).cuda())
        self.grid = Grid.for_scene(scene)
        self.t = 0
        self.queries = scene.n

    def step(self):
        from paper_cs_0608108_b300 import neighbor_energy
        x = self.frames[self.t % len(self.frames)].detach().requires_grad_(True)
        self.t += 1
        E = neighbor_energy(x, self.grid, self.scene.r)
        E.backward()
        self.last = (E, x)

    def check_graphs(self, rotation, outputs):
        """The replayed graphs give what the eager step gives, frame by frame
        (energy to 1e-12 relative, gradient to 1e-6 of its largest entry)."""
        import torch
        for f, gr in enumerate(rotation.graphs):
            gr.replay()
            torch.cuda.synchronize()
            Eg, xg = outputs[f]
            eg, gg = float(Eg.item()), xg.grad.detach().clone()
            self.t = f
            self.step()
            torch.cuda.synchronize()
            ee, ge = float(self.last[0].item()), self.last[1].grad
            if abs(eg - ee) > 1e-12 * max(abs(ee), 1e-300) or \
                    float((gg - ge).abs().max()) > 1e-6 * max(float(ge.abs().max()), 1e-30):
                raise SystemExit(f"walk graph of frame {f} differs from the eager step: E {eg} vs {ee}")
        self.t = 0

    def check(self):
        self.grid.sync()

    def algorithmic_bytes(self):
        n, C = self.scene.n, (1 << sum(self.scene.log2_cells)) + 1
        # energy walk: the points, their indices and the cell starts read;
        # adjoint walk: the same plus the gradient written (16 B a point)
        walk = 16 * n + 4 * n + 4 * C
        return {"k_reduce": walk, "k_reduce_eq2": walk, "k_reduce_grad": walk + 16 * n,
                "k_reduce_grad_eq2": walk + 16 * n, "k_bin_key": 24 * n + 8 * C,
                "k_bin_scatter": 48 * n + 4 * C}

    def step_bytes(self):
        n, C = self.scene.n, (1 << sum(self.scene.log2_cells)) + 1
        return 36 * n + 4 * C + 2 * (20 * n + 4 * C) + 16 * n


class BatchWork:
    """The batch of scenes in one library batch; params: the planner's
    choices (None: the ones tuned for this batch on a B300, from the
    package's cache, else the defaults)."""

    def __init__(self, scenes, graph=True, params="tuned"):
        import torch
        from paper_cs_0608108_b300 import Batch, Grid, lookup_batch_params
        self.scenes = scenes
        self.pos = [torch.from_numpy(s.pos).cuda() for s in scenes]
        self.offs = [torch.empty(s.n + 1, dtype=torch.int64, device="cuda") for s in scenes]
        # each scene's neighbor total, from the plain single-scene path
        self.totals = []
        for sc, p in zip(scenes, self.pos):
            g = Grid.for_scene(sc)
            g.build(p)
            off, _ = g.query_radius(sc.r)
            self.totals.append(int(off[-1].item()))
            g.close()
        self.ids = [torch.empty(max(t, 1), dtype=torch.int32, device="cuda") for t in self.totals]
        self.params = lookup_batch_params(scenes) if params == "tuned" else params
        self.batch = Batch(list(zip(scenes, self.pos)), self.offs, self.ids, params=self.params)
        self.graph = graph
        self.queries = sum(s.n for s in scenes)

    def step(self):
        self.batch.run(self.graph)

    def check(self):
        self.batch.sync()

    def algorithmic_bytes(self):
        return {"batch_graph": float(self.step_bytes())}

    def step_bytes(self):
        tot = 0
        for s, t in zip(self.scenes, self.totals):
            n, C = s.n, (1 << sum(s.log2_cells)) + 1
            tot += 36 * n + 4 * C + 20 * n + 4 * C + 8 * n + 4 * t
        return tot


class LoopWork(RadiusWork):
    """The plain single-scene path looped over the batch's scenes."""


# what each workload is (the `config.description` of both arms' lines)
DESC = {
    "radius_1m": "1M-point all-agents radius, 128^3 cyclic, r=1.5 cells, uniform + Gaussian mixture "
                 "(each scene's binning and query on a stream of its own)",
    "radius_uniform": "1M uniform all-agents radius, 128^3 cyclic, r=1.5 cells",
    "radius_mixture": "1M Gaussian-mixture all-agents radius, 128^3 cyclic, r=1.5 cells",
    "radius_mixture_250k": "250k Gaussian-mixture all-agents radius (16 components, the 1M mixture's density), "
                           "128^3 cyclic, r=1.5 cells",
    "radius_uniform_cube": "1M uniform, GPU bin-lattice cube scan",
    "radius_mixture_cube": "1M mixture, GPU bin-lattice cube scan",
    "radius_1m_cube": "same, GPU bin-lattice cube scan",
    "knn_4m": "4M-point K-nearest (K=16 and 64), 256^3, cyclic x,y, r_max=4 cells",
    "knn_4m_cube": "4M-point K-nearest (K=16 and 64), 256^3, cyclic x,y, r_max=4 cells, GPU bin-lattice walk",
    "knn_250k": "250k-point K-nearest (K=16 and 64) at the 4M configuration's density, 128x128x64, cyclic x,y, "
                "r_max=4 cells",
    "walk_1m": "1M-point random walk step: rebin + energy + adjoint, 128^3 cyclic, r=1.5 cells",
    "batched": "256 uneven scenes (log-uniform 1k-200k points), one graph replay",
    "batched_loop": "256 uneven scenes, plain path looped per scene",
    "tiny": "20k-point radius, 32^3 non-cyclic, r=0.96 cells",
    "terrain_1m": "1M agents on a bumpy terrain (z = 0.5 + 0.01 sin sin), 2% flying, 128^3, cyclic x, y, "
                  "r = 1.5 cells, classes walk",
    "terrain_1m_planes": "1M agents on a bumpy terrain (z = 0.5 + 0.01 sin sin), 2% flying, 128^3, cyclic x, y, "
                         "r = 1.5 cells, planes walk",
    "radius_far_20k": "20,480 uniform points, 64^3 cyclic (load 0.078), r = 24 cells, 100k uniform centers: "
                      "the volume comparison takes the non-empty list method",
    "radius_centers_1m": "1M Gaussian-mixture points, 128^3 cyclic, r=1.5 cells; 1M query centers, half from the "
                         "same mixture (another seed), half uniform",
}


def workload_config(name, world, queries):
    """The `config` of a bench line, the same for both arms of a workload."""
    return {"workload": name, "description": DESC.get(name, name), "l2": "flushed between steps",
            "queries_per_step": int(queries), "parallelism": f"replicas x{world}"}


def make_work(name):
    from paper_cs_0608108_b300 import synth
    if name == "radius_1m":
        return RadiusWork([synth.uniform_1m_scene(), synth.mixture_1m_scene()]), DESC[name]
    if name == "radius_uniform":
        return RadiusWork([synth.uniform_1m_scene()]), DESC[name]
    if name == "radius_mixture":
        return RadiusWork([synth.mixture_1m_scene()]), DESC[name]
    if name == "radius_mixture_250k":
        return RadiusWork([synth.mixture_250k_scene()]), DESC[name]
    if name == "radius_uniform_cube":
        return RadiusWork([synth.uniform_1m_scene()], "cube"), DESC[name]
    if name == "radius_mixture_cube":
        return RadiusWork([synth.mixture_1m_scene()], "cube"), DESC[name]
    if name == "radius_1m_cube":
        return RadiusWork([synth.uniform_1m_scene(), synth.mixture_1m_scene()], "cube"), DESC[name]
    if name == "knn_4m":
        return KnnWork(synth.knn_4m_scene()), DESC[name]
    if name == "knn_4m_cube":
        return KnnWork(synth.knn_4m_scene(), method="cube"), DESC[name]
    if name == "knn_250k":
        return KnnWork(synth.knn_250k_scene()), DESC[name]
    if name == "walk_1m":
        return WalkWork(synth.uniform_1m_scene()), DESC[name]
    if name == "batched":
        return BatchWork(synth.batched_scenes()), DESC[name]
    if name == "batched_loop":
        return LoopWork(synth.batched_scenes()), DESC[name]
    if name == "tiny":
        return RadiusWork([synth.tiny_scene()]), DESC[name]
    if name in ("terrain_1m", "terrain_1m_planes"):
        walk = "planes" if name.endswith("planes") else "classes"
        return RadiusWork([terrain_scene()], walk=walk), DESC[name]
    if name == "radius_far_20k":
        return CentersWork(make_work_scene_far(), synth.uniform_points(100_000, 0x51D00301)), DESC[name]
    if name == "radius_centers_1m":
        return CentersWork(synth.mixture_1m_scene(), centers_1m()), DESC[name]
    raise SystemExit(f"unknown workload {name}")


def terrain_scene():
    from paper_cs_0608108_b300 import synth
    return synth.Scene(synth.terrain_points(1_000_000, 0x51D00400), (0.0, 0.0, 0.0), 1.0 / 128, (7, 7, 7), 3,
                       1.5 / 128, "terrain_1m")


def make_work_scene_far():
    from paper_cs_0608108_b300 import synth
    return synth.Scene(synth.uniform_points(20_480, 0x51D00300), (0.0, 0.0, 0.0), 1.0 / 64, (6, 6, 6), 7,
                       24.0 / 64, "far_20k")


def centers_1m():
    """Query centers of the centers workload: 500k drawn from the points'
    mixture with another seed, 500k uniform, interleaved."""
    from paper_cs_0608108_b300 import synth
    a = synth.gaussian_mixture_points(500_000, synth.SEEDS["mixture_1m"] + 0x100)
    b = synth.uniform_points(500_000, synth.SEEDS["mixture_1m"] + 0x101)
    c = np.empty((1_000_000, 4), np.float32)
    c[0::2], c[1::2] = a, b
    return c


SWEEPS = {
    # the paper's sizes (Sec. IV.A, Fig. 9 and 10): 20,480 objects, 16^3 / 32^3 / 64^3
    "paper_20k": dict(n=20_480, m=100_000, log2=4, shifts=(0, 1, 2), d=(0.5, 1, 2, 3, 4, 6)),
    # the same loads on a 64x larger problem: 64^3 / 128^3 / 256^3
    "b300_1m": dict(n=1_310_720, m=250_000, log2=6, shifts=(0, 1, 2), d=(0.5, 1, 2, 3, 4)),
}


def run_sweep(reps=3):
    """Discretization sweep: for each problem size, cyclic mask (xyz, none),
    mode (all neighbors within d; the nearest within d) and distance d (in
    cells of the coarsest lattice), the time of binning + one query of m
    uniform centers on each lattice, and the fastest lattice (the tuner of
    the library)."""
    import torch
    from paper_cs_0608108_b300 import synth, tune_lattice
    out, total_q, total_ms, launches = {}, 0, 0.0, 0
    for name, S in SWEEPS.items():
        pos = torch.from_numpy(synth.uniform_points(S["n"], 0x51D00100 + S["log2"])).cuda()
        cen = torch.from_numpy(synth.uniform_points(S["m"], 0x51D00200 + S["log2"])).cuda()
        rows = []
        for mask in (7, 0):
            for mode, k in (("radius", 0), ("nearest", 1)):
                for d in S["d"]:
                    s0 = 1.0 / (1 << S["log2"])
                    ms, best = tune_lattice((0, 0, 0), s0, (S["log2"],) * 3, mask, pos, d * s0, S["shifts"],
                                            centers=cen, k=k, reps=reps)
                    rows.append({"mask": mask, "mode": mode, "d": d,
                                 "lattices": [1 << (S["log2"] + x) for x in S["shifts"]],
                                 "ms": [round(t, 4) if np.isfinite(t) else None for t in ms],
                                 "best": 1 << (S["log2"] + S["shifts"][best]),
                                 "queries_per_s_best": S["m"] / (ms[best] * 1e-3)})
                    total_q += S["m"]
                    total_ms += ms[best]
        out[name] = {"n": S["n"], "m": S["m"], "loads": [S["n"] / (1 << 3 * (S["log2"] + x)) for x in S["shifts"]],
                     "rows": rows}
    return out, total_q, total_ms


def slowest_rank_ms(ms_step: float, device: str = "cuda") -> float:
    """The job's step time: the slowest rank's (max over ranks; the rank's own
    time when there is one rank or no process group)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms_step
    t = torch.tensor([ms_step], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(queries_per_rank: int, world: int, ms_step: float) -> float:
    """Whole-job throughput: every rank serves its own replica of the workload."""
    return queries_per_rank * world / (ms_step * 1e-3)


def same_run_comparisons(steps, warmup, flush, local):
    """The comparisons the metric names, measured in the same run as the
    default line: the GPU bin-lattice cube scan on the same two 1M scenes,
    and the 256 uneven scenes served by the library's batched graph against
    the plain single-scene path looped over them (their lists checked equal,
    scene by scene).  Device times with CUDA events, L2 flushed per step."""
    import torch
    from paper_cs_0608108_b300 import synth
    out = {}
    with ClockSampler(local) as clk:
        cube = RadiusWork([synth.uniform_1m_scene(), synth.mixture_1m_scene()], "cube")
        for _ in range(2):
            cube.step()
        cube.check()
        g, _ = capture_step(cube)
        ms = time_steps(cube, steps, warmup, flush, g)
        out["radius_1m_cube"] = {"ms_per_step": float(np.mean(ms)), "queries_per_s": cube.queries / (np.mean(ms) * 1e-3),
                                 "description": "same scenes, GPU bin-lattice cube scan (bounding cube of the sphere)"}
        del g, cube
        torch.cuda.empty_cache()
        scenes = synth.batched_scenes()
        bw = BatchWork(scenes)
        ms_b = time_steps(bw, steps, warmup, flush)
        bw.check()
        bd = BatchWork(scenes, params=None)
        ms_d = time_steps(bd, steps, warmup, flush)
        bd.check()
        del bd
        lw = LoopWork(scenes)
        ms_l = time_steps(lw, steps, warmup, flush)
        lw.check()
        same = all(torch.equal(a, b) for a, b in zip(bw.offs, lw.off)) and \
            all(torch.equal(a[:t], b[:t]) for a, b, t in zip(bw.ids, lw.ids, bw.totals))
        out["batched"] = {"ms_per_step": float(np.mean(ms_b)), "queries_per_s": bw.queries / (np.mean(ms_b) * 1e-3),
                          "scenes": len(scenes), "points": bw.queries, "planner": bw.params or "defaults",
                          "description": "256 uneven scenes, one graph replay (fused short-list scenes, "
                                         "concurrent branches for long-list scenes), planner choices tuned "
                                         "on a B300 (package cache)"}
        out["batched_default_planner"] = {"ms_per_step": float(np.mean(ms_d)),
                                          "queries_per_s": bw.queries / (np.mean(ms_d) * 1e-3)}
        out["batched_loop"] = {"ms_per_step": float(np.mean(ms_l)), "queries_per_s": lw.queries / (np.mean(ms_l) * 1e-3),
                               "description": "the plain single-scene path called scene after scene"}
        out["batched_equals_loop"] = bool(same)
        del bw, lw
        torch.cuda.empty_cache()
    out["clocks"] = clk.summary()
    return out


def capture_step(work):
    """The step captured once in a CUDA graph (every call of the step is
    asynchronous once its tables and buffers are sized); returns the graph
    and the number of library kernels it holds."""
    import torch
    from paper_cs_0608108_b300 import launch_count
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        work.step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    l0 = launch_count()
    with torch.cuda.graph(graph):
        work.step()
    torch.cuda.synchronize()
    return graph, launch_count() - l0


class _Rotation:
    """Graphs replayed in turn (one per input frame of a rotating step)."""

    def __init__(self, graphs):
        self.graphs, self.k = graphs, 0

    def replay(self):
        self.graphs[self.k % len(self.graphs)].replay()
        self.k += 1


def capture_walk(work):
    """The walk step (rebin, energy, adjoint through autograd) captured once
    per input frame, the graphs replayed in the frames' order; returns the
    rotation and the library kernels one step holds."""
    import torch
    from paper_cs_0608108_b300 import launch_count
    graphs, outputs, per = [], [], 0
    for f in range(len(work.frames)):
        work.t = f
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            work.step()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        work.t = f
        gr = torch.cuda.CUDAGraph()
        l0 = launch_count()
        with torch.cuda.graph(gr):
            work.step()
        torch.cuda.synchronize()
        per = launch_count() - l0
        graphs.append(gr)
        outputs.append(work.last)
    work.t = 0
    rot = _Rotation(graphs)
    work.check_graphs(rot, outputs)
    return rot, per


def _barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def time_steps(work, steps, warmup, flush, graph=None):
    """Per-step device times (CUDA events on the launching stream, L2 flushed
    before each step); graph: replay it instead of calling the step.  The
    timed steps are bracketed by a device synchronisation and a barrier over
    the ranks on both sides."""
    import torch
    st = torch.cuda.current_stream()
    run = graph.replay if graph is not None else work.step
    for _ in range(warmup):
        run()
    work.check()
    torch.cuda.synchronize()
    _barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for a, b in evs:
        flush.zero_()                        # evict L2 between timed steps
        a.record(st)
        run()
        b.record(st)
    torch.cuda.synchronize()
    _barrier()
    return [a.elapsed_time(b) for a, b in evs]


# kernel name -> phase of the step (bin: keys, scatter and the order inside
# cells; scan: the prefix sums of the binning and of the list offsets; query:
# the walks and the cell kernels' tests; sort: the sorts of long lists;
# expand: the heavy cells' lists written from their hit masks)
_PHASE = (("expand", ("k_expand", "k_cell_expand")), ("sort", ("k_sort",)), ("scan", ("scan",)),
          ("bin", ("k_bin", "k_cell_order", "k_center_key", "k_center_scatter")))


def phase_split(rows, steps):
    """Milliseconds per step of each phase, from the per-kernel timing pass
    (kernels one after another, so the phases add up to more than a step in
    which streams overlap)."""
    if not rows:
        return None
    out = {}
    for name, (cnt, tot) in rows.items():
        ph = next((p for p, keys in _PHASE if any(k in name for k in keys)), "query")
        out[ph] = out.get(ph, 0.0) + tot / max(steps, 1)
    return {k: round(v, 4) for k, v in sorted(out.items())}


def step_rates(work, ms_step):
    """Queries, list entries (hits) and candidate pair tests per second of the
    timed step (the pair tests are the algorithmic ones: every candidate the
    walk of the method reaches; None where the workload does not count them)."""
    out = {"queries_per_s": work.queries / (ms_step * 1e-3)}
    hits = getattr(work, "totals", None)
    if hits is not None:
        out["hits_per_s"] = float(sum(hits)) / (ms_step * 1e-3)
    pairs = getattr(work, "step_pairs", None)
    if pairs is not None:
        p = pairs()
        if p:
            out["candidate_pairs_per_s"] = p / (ms_step * 1e-3)
    return out


def kernel_report(lib):
    buf = ctypes.create_string_buffer(1 << 16)
    lib.si_kernel_timing_report(buf, len(buf))
    rows = {}
    for line in buf.value.decode().splitlines():
        f = line.rsplit(" ", 2)
        if len(f) == 3:
            rows[f[0]] = (int(f[1]), float(f[2]))
    return rows


def _oracle_scene(name):
    from paper_cs_0608108_b300 import synth
    if name in ("radius_1m", "radius_1m_cube", "walk_1m", "radius_uniform", "radius_uniform_cube"):
        return synth.uniform_1m_scene()
    if name == "radius_mixture_250k":
        return synth.mixture_250k_scene()
    if name in ("radius_mixture", "radius_mixture_cube", "radius_centers_1m"):
        return synth.mixture_1m_scene()
    if name in ("knn_4m", "knn_4m_cube"):
        return synth.knn_4m_scene()
    if name == "knn_250k":
        return synth.knn_250k_scene()
    if name == "radius_far_20k":
        return make_work_scene_far()
    if name in ("terrain_1m", "terrain_1m_planes"):
        return terrain_scene()
    if name == "tiny":
        return synth.tiny_scene()
    return synth.batched_scenes()[0]


class OracleRunner:
    """The oracle (FP64 brute force over all points) as it stands, on bounded
    samples of the workload's query points, with every host thread."""

    def __init__(self, name):
        import oracle
        from paper_cs_0608108_b300 import synth
        self.oracle = oracle
        self.name = name
        # the workload's scenes (both of the two-scene step) and K values
        if name in ("radius_1m", "radius_1m_cube"):
            self.scs = [synth.uniform_1m_scene(), synth.mixture_1m_scene()]
        else:
            self.scs = [_oracle_scene(name)]
        self.sc = self.scs[0]
        self.knn = name in ("knn_4m", "knn_4m_cube", "knn_250k")
        self.ks = (16, 64) if self.knn else (None,)
        self.threads = oracle.max_threads()
        self.rng = np.random.default_rng(0)
        self.centers = centers_1m() if name == "radius_centers_1m" else None
        if name == "radius_far_20k":
            self.centers = synth.uniform_points(100_000, 0x51D00301)

    def queries_per_step(self):
        """The queries one step of the workload answers (as the GPU arm counts them)."""
        if self.centers is not None:
            return self.centers.shape[0]
        return sum(sc.n for sc in self.scs) * len(self.ks)

    def run(self, m):
        """Time m queries, split evenly over the workload's scenes and K values."""
        o = self.oracle
        parts = [(sc, k) for sc in self.scs for k in self.ks]
        t = 0.0
        for i, (sc, k) in enumerate(parts):
            mi = m // len(parts) + (1 if i < m % len(parts) else 0)
            if mi == 0:
                continue
            q = self.rng.choice(sc.n, mi, replace=False)
            t0 = time.perf_counter()
            if self.centers is not None:
                o.radius(sc.pos, self.centers[q], sc.box, sc.cyclic_mask, sc.r, None)
            elif self.knn:
                o.knn(sc.pos, sc.pos[q], sc.box, sc.cyclic_mask, k, sc.r, q)
            elif self.name == "walk_1m":
                o.reduce(sc.pos, q, sc.box, sc.cyclic_mask, sc.r)
            else:
                o.radius(sc.pos, sc.pos[q], sc.box, sc.cyclic_mask, sc.r, q)
            t += time.perf_counter() - t0
        return t

    def calibrate(self, seconds):
        m = max(64, self.threads * 32)   # the oracle hands out queries in chunks of 16
        self.run(m)                       # warm the thread pool
        dt = self.run(m)
        return int(min(self.sc.n, max(m, m * seconds / max(dt, 1e-4))))

    def describe(self, m, total_s, steps):
        what = "query centers" if self.centers is not None else "query points"
        scenes = " + ".join(f"{sc.n}-point {sc.name}" for sc in self.scs)
        ks = f", K = {' and '.join(str(k) for k in self.ks)}" if self.knn else ""
        return (f"{steps} x {m} random {what} of the workload ({scenes}{ks}, split evenly), "
                f"FP64 brute force over all points, {self.threads} threads, {total_s:.1f} s")


def tier_b(name):
    """The CPU cell walks of oracle/cells.c (FP64, every host thread) over the
    whole radius workload: binning plus every query's sorted list, for the
    spherical index (offset table + Eq. 1 cell test) and the bin-lattice cube
    scan.  None for workloads other than the all-agents radius scenes."""
    import oracle
    from paper_cs_0608108_b300 import synth
    scenes = {"radius_1m": [synth.uniform_1m_scene, synth.mixture_1m_scene],
              "radius_1m_cube": [synth.uniform_1m_scene, synth.mixture_1m_scene],
              "radius_uniform": [synth.uniform_1m_scene], "radius_uniform_cube": [synth.uniform_1m_scene],
              "radius_mixture": [synth.mixture_1m_scene], "radius_mixture_cube": [synth.mixture_1m_scene],
              "tiny": [synth.tiny_scene]}.get(name)
    if scenes is None:
        return None
    out = {"unit": "queries/s", "threads": oracle.max_threads(), "kind": "cpu cell walks (oracle/cells.c), FP64",
           "sample": "every query of " + " + ".join(f.__name__.replace("_scene", "") for f in scenes)
                     + ", binning included"}
    for method in ("sphere", "cube"):
        q, t = 0, 0.0
        for make in scenes:
            sc = make()
            t0 = time.perf_counter()
            oracle.cells_radius(sc.pos, sc.origin, sc.cell_size, sc.log2_cells, sc.cyclic_mask,
                                float(np.float32(sc.r)), method=method)
            t += time.perf_counter() - t0
            q += sc.n
        out[method] = {"value": q / t, "seconds": t}
    # one thread, on every 32nd query of each scene (binning included)
    one = {"threads": 1, "sample": "every 32nd query of each scene, binning of the whole scene included"}
    for method in ("sphere", "cube"):
        q, t = 0, 0.0
        for make in scenes:
            sc = make()
            sel = np.arange(0, sc.n, 32, dtype=np.int64)
            t0 = time.perf_counter()
            oracle.cells_radius(sc.pos, sc.origin, sc.cell_size, sc.log2_cells, sc.cyclic_mask,
                                float(np.float32(sc.r)), queries=sel, method=method, threads=1)
            t += time.perf_counter() - t0
            q += sel.shape[0]
        one[method] = {"value": q / t, "seconds": t}
    out["single_thread"] = one
    return out


def cpu_baseline(name, budget_s=15.0):
    r = OracleRunner(name)
    m = r.calibrate(budget_s)
    dt = r.run(m)
    cb = {"value": m / dt, "unit": "queries/s", "cores": r.threads, "kind": "oracle",
          "sample": r.describe(m, dt, 1)}
    tb = tier_b(name)
    if tb is not None:
        cb["tier_b"] = tb
    return cb


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="radius_1m")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="call the step eagerly instead of replaying its graph")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the same-run cube-scan and batched-vs-loop comparisons of the default workload")
    args = ap.parse_args()
    rank, world, local = dist_setup()
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        if rank != 0:
            return
        r = OracleRunner(args.workload)
        m = r.calibrate(min(4.0, 90.0 / max(args.steps + args.warmup, 1)))
        for _ in range(args.warmup):
            r.run(max(1, m // 4))
        total = sum(r.run(m) for _ in range(args.steps))
        v = m * args.steps / total
        cb = {"value": v, "unit": "queries/s", "cores": r.threads, "kind": "oracle",
              "sample": r.describe(m, total, args.steps)}
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": workload_config(args.workload, args.gpus, r.queries_per_step()),
                "cpu_baseline": cb,
                "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    torch.cuda.set_device(local)
    if args.workload == "sweep":
        if rank != 0:
            return
        from paper_cs_0608108_b300 import launch_count
        l0 = launch_count()
        with ClockSampler(local) as clk:
            table, q, ms_tot = run_sweep()
        line = {"metric": "discretization sweep: queries/s of the fastest lattice per point (Fig. 9/10 shape)",
                "value": q / (ms_tot * 1e-3), "unit": "queries/s", "n_gpus": 1, "steps": 1, "warmup": 1,
                "ms_per_step": ms_tot, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": "sweep", "description": "uniform objects and centers in the unit cube; "
                           "binning + one query per timed round, median of 3 rounds", "l2": "not flushed"},
                "gpu_launches": int(launch_count() - l0), "clocks": clk.summary(), "roofline": None,
                "e2e": None, "sweep": table}
        print(json.dumps(line))
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_cs_0608108_b300 import _native, launch_count
    lib = _native.lib()
    work, _ = make_work(args.workload)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    # whole-step timing (no per-kernel events)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # the query workloads replay the step as one CUDA graph (the batched path
    # does the same inside the library); the plain-path loop stays eager
    use_graph = (not args.no_graph and isinstance(work, (RadiusWork, CentersWork, KnnWork, WalkWork))
                 and not isinstance(work, LoopWork))
    graph, graph_launches = None, 0
    if use_graph:
        for _ in range(2):
            work.step()
        work.check()
        if isinstance(work, WalkWork):
            graph, graph_launches = capture_walk(work)
        else:
            graph, graph_launches = capture_step(work)
    l0 = launch_count()
    with ClockSampler(local) as clk:
        ms = time_steps(work, args.steps, args.warmup, flush, graph)
    launches = graph_launches if use_graph else (launch_count() - l0) // (args.steps + args.warmup)
    work.check()
    ms_step = slowest_rank_ms(float(np.mean(ms)))
    value = job_value(work.queries, world, ms_step)
    # per-kernel timing pass (CUDA events around each launch, same stream);
    # the library and the scenes run their kernels one after another here,
    # so each launch is timed alone (the shares then compare with the ncu
    # launch list, which serialises launches too)
    lib.si_kernel_timing_enable(1)
    if hasattr(work, "serial"):
        work.serial = True
    kernel_report(lib)
    time_steps(work, args.steps, 1, flush)
    rows = kernel_report(lib)
    lib.si_kernel_timing_enable(0)
    if hasattr(work, "serial"):
        work.serial = False
    alg = work.algorithmic_bytes()
    peak, peak_kind = peaks()
    from paper_cs_0608108_b300 import measure_pair_rate
    pair_peak = measure_pair_rate(True)
    dom = max(rows.items(), key=lambda kv: kv[1][1])[0] if rows else None
    roof = None
    if dom is not None:
        cnt, tot = rows[dom]
        avg_ms = tot / max(cnt, 1)
        a_bytes = alg.get(dom)
        achieved = (a_bytes / (avg_ms * 1e-3) / 1e9) if a_bytes else None
        share = {k: round(v[1] / sum(x[1] for x in rows.values()), 4)
                 for k, v in sorted(rows.items(), key=lambda kv: -kv[1][1])}
        traffic = ncu_traffic(dom, args.workload)
        pairs = work.algorithmic_pairs().get(dom) if hasattr(work, "algorithmic_pairs") else None
        # the HBM roofline of the dominant kernel (its algorithmic bytes per
        # launch over its mean launch time), the whole step's, and the pair
        # tests of the kernel against the measured pair-test rate of this GPU
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": a_bytes, "avg_launch_ms": avg_ms, "traffic": traffic,
                "traffic_over_algorithmic": (traffic / a_bytes) if (traffic and a_bytes) else None,
                "kernel_share": share}
        if pairs:
            ach = pairs / (avg_ms * 1e-3)
            roof["alu"] = {"achieved": ach, "peak": pair_peak, "unit": "pair tests/s",
                           "frac": (ach / pair_peak) if pair_peak else None,
                           "peak_kind": "measured: si_measure_pair_rate, packed f32x2 pair tests, best of 5",
                           "algorithmic_pairs_per_launch": pairs}
    step_gbs = work.step_bytes() / (ms_step * 1e-3) / 1e9
    rates = step_rates(work, ms_step)
    phases = phase_split(rows, args.steps)
    if roof is not None:
        roof["step"] = {"achieved": step_gbs, "frac": step_gbs / peak, "unit": "GB/s",
                        "algorithmic_bytes": work.step_bytes()}
    e2e = None
    if not args.no_e2e and isinstance(work, RadiusWork):
        # through the C ABI's host-buffer call (the headline e2e), then the
        # same copies pipelined across steps through the Python API (context)
        e_ms, e_wall, bi, bo = e2e_radius_host(work, max(3, args.steps // 2), 2)
        e_ms = slowest_rank_ms(e_ms)
        p_ms, _, _ = e2e_radius(work, max(3, args.steps // 2), 2)
        p_ms = slowest_rank_ms(p_ms)
        e2e = {"value": job_value(work.queries, world, e_ms), "unit": "queries/s",
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "ms_per_step": e_ms,
               "host_wall_ms_per_step": e_wall,
               "call": "si_query_radius_host per scene, a host thread each (page-locked host buffers in and out)",
               "pipelined": {"value": job_value(work.queries, world, p_ms), "ms_per_step": p_ms,
                             "how": "torch copies on a second stream, a step's lists copied out while the "
                                    "next step's points come in"}}
        # the host link's own bound for these bytes (each direction alone)
        link = host_link()
        link["copy_bound_ms_per_step"] = (bi / link["h2d_gbs"] + bo / link["d2h_gbs"]) / 1e6
        link["d2h_bound_ms_per_step"] = bo / link["d2h_gbs"] / 1e6
        e2e["host_link"] = link
    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": workload_config(args.workload, world, work.queries),
            "step": ("library calls" if not use_graph else
                     "one CUDA graph replay of the autograd step (rebin, energy, adjoint), a graph per input frame"
                     if isinstance(work, WalkWork) else "one CUDA graph replay of the library calls"),
            "step_algorithmic_gbs": step_gbs, "step_hbm_frac": step_gbs / peak,
            "roofline": roof, "gpu_launches": int(launches), "clocks": clk.summary(), "e2e": e2e,
            "rates": rates, "phases_ms_per_step": phases,
            "ms_samples": {"median": float(np.median(ms)), "min": float(np.min(ms)),
                           "max": float(np.max(ms))}}
    if args.workload == "radius_1m" and not args.no_compare:
        cmp = same_run_comparisons(max(3, min(args.steps, 10)), 3, flush, local)
        cmp["sphere_vs_cube"] = cmp["radius_1m_cube"]["ms_per_step"] / ms_step
        cmp["batched_vs_loop"] = cmp["batched_loop"]["ms_per_step"] / cmp["batched"]["ms_per_step"]
        line["comparisons"] = cmp
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

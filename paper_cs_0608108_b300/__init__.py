"""B300 spherical-index neighborhood queries (Brodu, "Spherical Indexing for
Neighborhood Queries").

Thin Python layer over the C ABI of include/si.h: it only marshals torch
device tensors and the current CUDA stream into the library's calls.  Every
step of binning, querying, sorting and reducing runs in the library's CUDA
kernels; there is no CPU path.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import math
import os

import torch

from . import _native as N

__all__ = ["Grid", "NeighborEnergy", "neighbor_energy", "Batch", "launch_count", "tune_lattice"]


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


def _check_points(pos: torch.Tensor) -> torch.Tensor:
    if not (pos.is_cuda and pos.dtype == torch.float32 and pos.dim() == 2 and pos.shape[1] == 4):
        raise ValueError("points must be a CUDA float32 tensor of shape (n, 4)")
    return pos.contiguous()


def _check_out(t, dtype, numel, what):
    """A caller-given output buffer must be a contiguous CUDA tensor of the
    right type holding at least `numel` elements (the library writes there)."""
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and t.numel() >= numel):
        raise ValueError(f"{what} must be a contiguous CUDA {dtype} tensor with at least {numel} elements")


def _centers(centers):
    """(tensor whose pointer is passed, m) for a centers argument.  A NULL
    pointer means all agents, so an empty centers tensor passes a one-row
    buffer (never read) with m = 0."""
    c = _check_points(centers)
    if c.shape[0] == 0:
        return torch.zeros((1, 4), dtype=torch.float32, device=c.device), 0
    return c, c.shape[0]


class _CudaArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 2}


def _device_view(ptr, shape, typestr) -> torch.Tensor:
    """Zero-copy torch view of library-owned device memory."""
    if int(torch.Size(shape).numel()) == 0:
        return torch.empty(shape, dtype={"<i4": torch.int32, "<f4": torch.float32}[typestr], device="cuda")
    return torch.as_tensor(_CudaArray(ptr, shape, typestr), device="cuda")


def launch_count() -> int:
    """Kernel launches issued by the library so far in this process."""
    return int(N.lib().si_launch_count())


def measure_pair_rate(packed: bool = True) -> float:
    """Measured pair tests per second of the current device (the arithmetic
    roofline of the radius kernels): packed f32x2 or scalar FP32 form."""
    out = ctypes.c_double(0.0)
    N.check(N.lib().si_measure_pair_rate(1 if packed else 0, ctypes.byref(out)), "si_measure_pair_rate")
    return out.value


def make_desc(origin, cell_size, log2_cells, cyclic_mask, r_max) -> N.GridDesc:
    d = N.GridDesc()
    for a in range(3):
        d.origin[a] = float(origin[a])
        d.log2_cells[a] = int(log2_cells[a])
    d.cell_size = float(cell_size)
    d.cyclic_mask = int(cyclic_mask)
    d.r_max = float("inf") if r_max is None else float(r_max)
    return d


def tune_lattice(origin, cell_size, log2_cells, cyclic_mask, pos: torch.Tensor, r: float, shifts,
                 centers=None, k: int = 0, reps: int = 5):
    """Time binning + one query (radius r, or the k nearest within r) on the
    region cut 2^shift times finer per axis, for each shift.  Returns
    (milliseconds per round for each shift, inf where invalid; index of the
    fastest)."""
    pos = _check_points(pos)
    d = make_desc(origin, cell_size, log2_cells, cyclic_mask, r)
    m = pos.shape[0]
    c = None
    if centers is not None:
        c, m = _centers(centers)
    sh = (ctypes.c_int32 * len(shifts))(*[int(x) for x in shifts])
    ms = (ctypes.c_float * len(shifts))()
    best = ctypes.c_int32(-1)
    N.check(N.lib().si_tune_lattice(ctypes.byref(d), _ptr(pos), pos.shape[0], _ptr(c), m, float(r), int(k),
                                    sh, len(shifts), int(reps), ms, ctypes.byref(best), _stream()),
            "si_tune_lattice")
    return [float(x) for x in ms], int(best.value)


class Grid:
    """A power-of-two cubic-cell lattice with its offset tables (Sec. II) and
    the binned points of the last `build`."""

    def __init__(self, origin, cell_size, log2_cells, cyclic_mask, r_max, capacity: int):
        self._lib = N.lib()
        self.desc = make_desc(origin, cell_size, log2_cells, cyclic_mask, r_max)
        h = ctypes.c_void_p()
        N.check(self._lib.si_grid_create(ctypes.byref(self.desc), int(capacity), ctypes.byref(h)),
                "si_grid_create")
        self._h = h
        self.capacity = int(capacity)
        self.n = 0
        self._pos = None
        self._ids_cap = 0
        self.build_id = 0

    @classmethod
    def for_scene(cls, scene, r_max=None, capacity=None):
        return cls(scene.origin, scene.cell_size, scene.log2_cells, scene.cyclic_mask,
                   scene.r if r_max is None else r_max, scene.n if capacity is None else capacity)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.si_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build(self, pos: torch.Tensor) -> "Grid":
        pos = _check_points(pos)
        N.check(self._lib.si_grid_build(self._h, _ptr(pos), pos.shape[0], _stream()), "si_grid_build")
        self._pos = pos          # keep the input alive while the grid refers to it
        self.n = pos.shape[0]
        self.build_id += 1
        return self

    def sync(self) -> None:
        N.check(self._lib.si_grid_sync(self._h, _stream()), "si_grid_sync")

    def info(self) -> dict:
        inf = N.GridInfo()
        N.check(self._lib.si_grid_get_info(self._h, ctypes.byref(inf)), "si_grid_get_info")
        return {k: getattr(inf, k) for k, _ in N.GridInfo._fields_}

    def cell_arrays(self):
        """(cell_start int32[n_cells+1], sorted points float32[n,4], perm int32[n]):
        copies of the grid's device arrays, for tests and tools."""
        inf = self.info()
        start = _device_view(inf["d_cell_start"], (inf["n_cells"] + 1,), "<i4").clone()
        spos = _device_view(inf["d_sorted_pos"], (inf["n"], 4), "<f4").clone()
        perm = _device_view(inf["d_perm"], (inf["n"],), "<i4").clone()
        return start, spos, perm

    # -- queries -------------------------------------------------------------
    def query_radius(self, r: float, include_self: bool = False, method: str = "sphere",
                     sort: bool = True, out_offsets=None, out_ids=None, sync_total: bool = True,
                     walk: str = "classes", centers=None, groups: bool = True):
        """Radius query.  Returns (offsets int64[m+1], ids int32[total]).
        centers None: all agents (query k is point k, m = n); else a CUDA
        float32 (m, 4) tensor of query centers.  method "sphere" (spherical
        index, switching to the list method when the volume comparison says
        it is cheaper), "sphere_only" (never switching), "cube" (bin-lattice
        scan) or "list" (non-empty list: every object tested); walk "classes"
        (sub-cell class tables), "paper" (Sec. III.A 64 tables) or "planes"
        (stacked z-planes, Sec. V); groups False serves every crowded cell
        on its own (same lists)."""
        if method not in ("sphere", "sphere_only", "cube", "list"):
            raise ValueError(f"unknown method {method!r}")
        flags = (N.SI_INCLUDE_SELF if include_self else 0) | (0 if sort else N.SI_NO_SORT) | \
                {"sphere": 0, "sphere_only": N.SI_SPHERE_ONLY, "cube": N.SI_METHOD_CUBE,
                 "list": N.SI_METHOD_LIST}[method] | \
                (N.SI_WALK_PAPER if walk == "paper" else 0) | (N.SI_WALK_PLANES if walk == "planes" else 0) | \
                (0 if groups else N.SI_NO_GROUPS)
        dev = self._pos.device
        m = self.n
        if centers is not None:
            centers, m = _centers(centers)
        off = out_offsets if out_offsets is not None else torch.empty(m + 1, dtype=torch.int64, device=dev)
        _check_out(off, torch.int64, m + 1, "out_offsets")
        if out_ids is not None:
            _check_out(out_ids, torch.int32, 0, "out_ids")
        ids = out_ids
        if ids is None:
            cap = self._ids_cap or max(16 * m, 1024)
            ids = torch.empty(cap, dtype=torch.int32, device=dev)
        total = ctypes.c_int64(0)
        st = self._lib.si_query_radius(self._h, _ptr(centers), m, float(r), flags, _ptr(off), _ptr(ids),
                                       ids.numel(), ctypes.byref(total) if sync_total else None,
                                       _stream())
        if st == N.SI_ERR_CAPACITY and out_ids is None:
            ids = torch.empty(max(int(total.value), 1), dtype=torch.int32, device=dev)
            st = self._lib.si_query_radius(self._h, _ptr(centers), m, float(r), flags, _ptr(off),
                                           _ptr(ids), ids.numel(), ctypes.byref(total), _stream())
        N.check(st, "si_query_radius")
        if sync_total:
            self._ids_cap = max(self._ids_cap, int(total.value))
            return off, ids[: int(total.value)]
        return off, ids

    def set_method(self, list_weight: float = 1.2, cube_below: float = 0.0, knn_cube_below: float = 0.0) -> "Grid":
        """Run-time method selection (si_grid_set_method, the Appendix's
        weighting factor and reversal distances): the list method is taken
        when list_weight times its estimated cost is below the sphere's
        (inf: never, 0: always); radius queries with r below cube_below cell
        sides, and K-nearest queries with r_max below knn_cube_below, take
        the bin lattice.  The results do not change."""
        N.check(self._lib.si_grid_set_method(self._h, float(list_weight), float(cube_below), float(knn_cube_below)),
                "si_grid_set_method")
        return self

    def query_radius_host(self, h_pos: torch.Tensor, r: float, h_offsets: torch.Tensor, h_ids: torch.Tensor,
                          include_self: bool = False, sort: bool = True) -> int:
        """End to end with host buffers (si_query_radius_host): h_pos, a CPU
        float32 (n, 4) tensor (page-locked for a direct copy), is copied to
        the device, binned and queried for all agents; the CSR result lands in
        the CPU tensors h_offsets (int64, n + 1) and h_ids (int32, its length
        is the capacity).  Returns the number of ids; raises when they do not
        fit."""
        if h_pos.device.type != "cpu" or h_pos.dtype != torch.float32 or h_pos.dim() != 2 or h_pos.shape[1] != 4:
            raise ValueError("h_pos must be a CPU float32 (n, 4) tensor")
        if not h_pos.is_contiguous():
            raise ValueError("h_pos must be contiguous")
        n = h_pos.shape[0]
        for t, dt, want in ((h_offsets, torch.int64, n + 1), (h_ids, torch.int32, 0)):
            if t.device.type != "cpu" or t.dtype != dt or not t.is_contiguous() or t.numel() < want:
                raise ValueError("h_offsets must be CPU int64 (n + 1); h_ids CPU int32, contiguous")
        flags = (N.SI_INCLUDE_SELF if include_self else 0) | (0 if sort else N.SI_NO_SORT)
        total = ctypes.c_int64(0)
        N.check(self._lib.si_query_radius_host(self._h, h_pos.data_ptr(), n, float(r), flags, h_offsets.data_ptr(),
                                               h_ids.data_ptr(), h_ids.numel(), ctypes.byref(total), _stream()),
                "si_query_radius_host")
        self.n = n
        if self._pos is None:   # the grid now holds the uploaded points; outputs go to this device
            self._pos = torch.empty((0, 4), dtype=torch.float32, device=torch.device("cuda", torch.cuda.current_device()))
        return int(total.value)

    def query_knn(self, k: int, r_max=None, include_self: bool = False, with_d2: bool = True,
                  out=None, centers=None, fast_d2: bool = False, method: str = "sphere"):
        """K nearest within r_max (None = grid's whole region), for every point
        (centers None) or for each row of a CUDA float32 (m, 4) tensor of
        query centers.  Returns (ids int32[m,k] padded -1, d2 float32[m,k]
        or None, counts int32[m]).  d2 is the FP32 rounding of the canonical
        FP64 squared distance; fast_d2 reports the kernel's FP32 value.
        method "cube": the bin-lattice walk (same results)."""
        dev = self._pos.device
        m = self.n
        if centers is not None:
            centers, m = _centers(centers)
        if out is None:
            ids = torch.empty((m, k), dtype=torch.int32, device=dev)
            d2 = torch.empty((m, k), dtype=torch.float32, device=dev) if with_d2 else None
            cnt = torch.empty(m, dtype=torch.int32, device=dev)
        else:
            ids, d2, cnt = out
            _check_out(ids, torch.int32, m * k, "out ids")
            _check_out(cnt, torch.int32, m, "out counts")
            if d2 is not None:
                _check_out(d2, torch.float32, m * k, "out d2")
        rm = float("inf") if r_max is None else float(r_max)
        if method not in ("sphere", "cube"):
            raise ValueError(f"unknown method {method!r}")
        flags = (N.SI_INCLUDE_SELF if include_self else 0) | (N.SI_FAST_D2 if fast_d2 else 0) | \
                (N.SI_METHOD_CUBE if method == "cube" else 0)
        N.check(self._lib.si_query_knn(self._h, _ptr(centers), m, int(k), rm, flags, _ptr(ids), _ptr(d2),
                                       _ptr(cnt), _stream()), "si_query_knn")
        return ids, d2, cnt

    def neighbor_reduce(self, r: float, energy=None, grad=None, grad_scale=None):
        """Fused smooth-kernel sum over radius neighbors: energy (float64[1]) and,
        when `grad` is given (float32[n,4]), dE/dx in input order."""
        if energy is not None:
            _check_out(energy, torch.float64, 1, "energy")
        if grad is not None:
            _check_out(grad, torch.float32, 4 * self.n, "grad")
        if grad_scale is not None:
            _check_out(grad_scale, torch.float32, 1, "grad_scale")
        N.check(self._lib.si_neighbor_reduce(self._h, float(r), N.SI_KERNEL_POLY6_CUBED, _ptr(energy),
                                             _ptr(grad), _ptr(grad_scale), _stream()),
                "si_neighbor_reduce")
        return energy, grad


class NeighborEnergy(torch.autograd.Function):
    """E(x) = sum_i sum_{j != i, |x_i - x_j| < r} (1 - |x_i - x_j|^2 / r^2)^3.

    forward bins the points and runs the energy kernel; backward runs the
    hand-written adjoint kernel, which walks the same neighborhoods and writes
    grad_output * dE/dx directly (the scale is read on the device)."""

    @staticmethod
    def forward(ctx, pos, grid: Grid, r: float):
        grid.build(pos.detach())
        energy = torch.empty(1, dtype=torch.float64, device=pos.device)
        grid.neighbor_reduce(r, energy=energy)
        ctx.grid, ctx.r, ctx.build_id = grid, r, grid.build_id
        return energy[0]

    @staticmethod
    def backward(ctx, g_out):
        if g_out is None or not ctx.needs_input_grad[0]:
            return None, None, None
        if ctx.grid.build_id != ctx.build_id:
            raise RuntimeError("the grid was rebuilt between forward and backward")
        scale = g_out.detach().to(torch.float32).reshape(1).contiguous()
        out = torch.empty((ctx.grid.n, 4), dtype=torch.float32, device=scale.device)
        ctx.grid.neighbor_reduce(ctx.r, energy=None, grad=out, grad_scale=scale)
        return out, None, None


def neighbor_energy(pos: torch.Tensor, grid: Grid, r: float) -> torch.Tensor:
    return NeighborEnergy.apply(pos, grid, r)


def _scene_array(scenes, offsets, ids, keep):
    arr = (N.SceneDesc * len(scenes))()
    for k, (sc, pos) in enumerate(scenes):
        pos = _check_points(pos)
        keep.append(pos)
        arr[k].desc = make_desc(sc.origin, sc.cell_size, sc.log2_cells, sc.cyclic_mask, sc.r)
        arr[k].d_pos = pos.data_ptr()
        arr[k].n = pos.shape[0]
        arr[k].r = float(sc.r)
        arr[k].d_offsets = offsets[k].data_ptr()
        arr[k].d_ids = ids[k].data_ptr()
        arr[k].ids_capacity = ids[k].numel()
    keep += list(offsets) + list(ids)
    return arr


def default_batch_params() -> dict:
    """The batch planner's defaults (si_batch_default_params)."""
    p = N.BatchParams()
    N.check(N.lib().si_batch_default_params(ctypes.byref(p)), "si_batch_default_params")
    return {"heavy_hits": p.heavy_hits, "q_tile": p.q_tile, "branches": p.branches,
            "blocks_per_sm": p.blocks_per_sm}


def _params(d) -> N.BatchParams:
    return N.BatchParams(float(d["heavy_hits"]), int(d["q_tile"]), int(d["branches"]), int(d["blocks_per_sm"]))


class Batch:
    """Many independent scenes served by one fixed set of launches; params
    (a dict of si_batch_params fields, None = defaults) sets the planner's
    choices, e.g. the ones tune_batch found."""

    def __init__(self, scenes, offsets, ids, flags: int = 0, params=None):
        self._lib = N.lib()
        self._keep = []
        arr = _scene_array(scenes, offsets, ids, self._keep)
        self.n_scenes = len(scenes)
        h = ctypes.c_void_p()
        prm = _params(params) if params is not None else None
        N.check(self._lib.si_batch_create_params(arr, len(scenes), int(flags),
                                                 ctypes.byref(prm) if prm is not None else None, ctypes.byref(h)),
                "si_batch_create_params")
        self._h = h

    def run(self, use_graph: bool = False):
        N.check(self._lib.si_batch_run(self._h, int(use_graph), _stream()), "si_batch_run")

    def sync(self):
        tot = (ctypes.c_int64 * self.n_scenes)()
        N.check(self._lib.si_batch_sync(self._h, tot, _stream()), "si_batch_sync")
        return list(tot)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.si_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Batch planner tuning with a cache on disk
# ---------------------------------------------------------------------------
def batch_scene_key(scene) -> tuple:
    """What the planner's choices depend on for one scene: its point count
    (bucket: rounded log2), its lattice (log2 cells per axis), its radius in
    cells (to a quarter cell), its load (points per cell, bucket: rounded
    2 log2) and its cyclic mask."""
    n = int(scene.n)
    cells = 1 << sum(scene.log2_cells)
    d = float(scene.r) / float(scene.cell_size)
    load = n / cells
    return (int(round(math.log2(n))) if n > 0 else -1, tuple(int(w) for w in scene.log2_cells),
            round(d * 4) / 4, int(round(2 * math.log2(load))) if load > 0 else -99, int(scene.cyclic_mask))


def batch_signature(scenes, flags: int = 0) -> str:
    """Cache key of a batch: the sorted multiset of its scenes' keys (the
    order of the scenes does not matter) and the flags."""
    keys = sorted(batch_scene_key(sc) for sc in scenes)
    return hashlib.sha1(repr((int(flags), keys)).encode()).hexdigest()


DEFAULT_CANDIDATES = [{"heavy_hits": h, "q_tile": t, "branches": b, "blocks_per_sm": 2048 // t // 2}
                      for h in (0.0, 4.0, 8.0, 16.0, 24.0, 64.0) for t in (64, 128, 256) for b in (8, 24)]


TUNING_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch_tuning.json")


def lookup_batch_params(scenes, cache: str = TUNING_CACHE, flags: int = 0):
    """The cached planner choices for these scenes (Scene objects), or None;
    times nothing.  The package's cache holds choices tuned on a B300."""
    if not cache or not os.path.exists(cache):
        return None
    with open(cache) as fh:
        store = json.load(fh)
    hit = store.get(batch_signature(scenes, flags))
    return dict(hit["params"]) if hit else None


def tune_batch(scenes, offsets, ids, flags: int = 0, cache: str | None = None, candidates=None,
               reps: int = 3):
    """The planner choices for these scenes ((scene, pos) pairs, outputs as
    for Batch): looked up in the JSON cache file `cache` by batch_signature,
    else timed by si_batch_tune over the candidates (default: the heavy-list
    threshold 0 / 4 / 8 / 16 / 24 / 64, query tile 64 / 128 / 256, 8
    branches) and stored there.  Returns (params dict, {"ms": [...] or None, "cached": bool,
    "signature": str})."""
    sig = batch_signature([sc for sc, _ in scenes], flags)
    store = {}
    if cache and os.path.exists(cache):
        with open(cache) as fh:
            store = json.load(fh)
        if sig in store:
            return dict(store[sig]["params"]), {"ms": None, "cached": True, "signature": sig}
    cands = list(candidates or DEFAULT_CANDIDATES)
    keep = []
    arr = _scene_array(scenes, offsets, ids, keep)
    carr = (N.BatchParams * len(cands))(*[_params(c) for c in cands])
    ms = (ctypes.c_float * len(cands))()
    best = ctypes.c_int32(-1)
    N.check(N.lib().si_batch_tune(arr, len(scenes), int(flags), carr, len(cands), int(reps), ms, ctypes.byref(best)),
            "si_batch_tune")
    params = dict(cands[best.value])
    if cache:
        store[sig] = {"params": params, "ms": float(ms[best.value]), "scenes": len(scenes)}
        tmp = cache + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(store, fh, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return params, {"ms": [float(x) for x in ms], "cached": False, "signature": sig}

"""CPU oracle for the neighborhood queries of Brodu, "Spherical Indexing for
Neighborhood Queries".

TEST INFRASTRUCTURE ONLY.  Only the tests, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline / reference legs may import, call or link anything
in this package.  It shares no code with the CUDA path and never imports it.

* `brute.c` (built into `_brute.so` by `build()`): FP64 brute force over all
  objects -- the plain definition of the query (Sec. I, Sec. II.A) -- and
  the same reduction through a plain bin lattice (cells at least r wide,
  3 x 3 x 3 cells per object), for sizes where O(n^2) is too slow.
* `cells.c` (in the same library): the radius query through CPU cell walks,
  the bin-lattice cube scan and the spherical index (Sec. II.A offset table
  by minimum bound, Sec. III.A Eq. 1 cell test), FP64: the timed CPU
  baselines of the cell methods, checked against the brute force.
* `sphere_index.py`: the paper's own method restated on the CPU in float64
  (tables of Sec. II.A and Sec. III.A, cell locations of Sec. II.B).  Used to
  pin the brute force against an independent algorithm and to check the
  paper's printed examples.

Every function here is pinned by tests under `tests/` against values the
paper prints, closed forms, invariants and scipy's periodic k-d tree.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_brute.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile brute.c and cells.c with gcc (no FMA contraction, OpenMP)."""
    srcs = [os.path.join(_HERE, f) for f in ("brute.c", "cells.c")]
    if force or not os.path.exists(_SO) or any(os.path.getmtime(_SO) < os.path.getmtime(f) for f in srcs):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-fopenmp", *srcs, "-o", _SO, "-lm"])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.or_canon_d2.restype = D
        lib.or_canon_d2.argtypes = [P, P, P, I32]
        lib.or_max_threads.restype = I32
        lib.or_radius_counts.argtypes = [P, I64, P, I64, P, P, I32, D, P, I32]
        lib.or_radius_lists.argtypes = [P, I64, P, I64, P, P, I32, D, P, P, I32]
        lib.or_knn.argtypes = [P, I64, P, I64, P, P, I32, D, I32, P, P, P, I32]
        lib.or_reduce.argtypes = [P, I64, P, I64, P, I32, D, P, P, I32]
        lib.or_reduce_cells.argtypes = [P, I64, P, I32, D, P, P, I32]
        lib.or_cells_radius.argtypes = [P, I64, P, D, P, I32, D, I32, P, I64, P, P, P, I32]
        _lib = lib
    return _lib


def _f4(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 4:
        raise ValueError("points must be float32 (n, 4)")
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def max_threads() -> int:
    return int(_load().or_max_threads())


def canon_d2(p, q, box, cyclic_mask: int) -> float:
    p = np.ascontiguousarray(np.asarray(p, np.float32).reshape(4))
    q = np.ascontiguousarray(np.asarray(q, np.float32).reshape(4))
    L = np.ascontiguousarray(box, dtype=np.float64)
    return float(_load().or_canon_d2(_ptr(p), _ptr(q), _ptr(L), int(cyclic_mask)))


def _self(self_idx, m):
    if self_idx is None:
        return None
    s = np.ascontiguousarray(self_idx, dtype=np.int64)
    assert s.shape == (m,)
    return s


def radius(pos, centers, box, cyclic_mask: int, r: float, self_idx=None, threads: int = 0):
    """All objects with canonical D^2 <= r^2 of each center, ids ascending.
    Returns (offsets int64[m+1], ids int32[total])."""
    lib = _load()
    pos, centers = _f4(pos), _f4(centers)
    n, m = pos.shape[0], centers.shape[0]
    L = np.ascontiguousarray(box, dtype=np.float64)
    s = _self(self_idx, m)
    counts = np.zeros(m, dtype=np.int64)
    lib.or_radius_counts(_ptr(pos), n, _ptr(centers), m, _ptr(s), _ptr(L), int(cyclic_mask),
                         float(r), _ptr(counts), int(threads))
    offsets = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    ids = np.zeros(int(offsets[-1]), dtype=np.int32)
    lib.or_radius_lists(_ptr(pos), n, _ptr(centers), m, _ptr(s), _ptr(L), int(cyclic_mask),
                        float(r), _ptr(offsets), _ptr(ids), int(threads))
    return offsets, ids


def radius_counts(pos, centers, box, cyclic_mask: int, r: float, self_idx=None, threads: int = 0):
    lib = _load()
    pos, centers = _f4(pos), _f4(centers)
    n, m = pos.shape[0], centers.shape[0]
    L = np.ascontiguousarray(box, dtype=np.float64)
    s = _self(self_idx, m)
    counts = np.zeros(m, dtype=np.int64)
    lib.or_radius_counts(_ptr(pos), n, _ptr(centers), m, _ptr(s), _ptr(L), int(cyclic_mask),
                         float(r), _ptr(counts), int(threads))
    return counts


def knn(pos, centers, box, cyclic_mask: int, k: int, r_max: float | None, self_idx=None,
        threads: int = 0):
    """K nearest within r_max (None = unbounded) by (D^2, id).
    Returns (ids int32[m,k] padded -1, d2 float64[m,k] padded inf, counts int32[m])."""
    lib = _load()
    pos, centers = _f4(pos), _f4(centers)
    n, m = pos.shape[0], centers.shape[0]
    L = np.ascontiguousarray(box, dtype=np.float64)
    s = _self(self_idx, m)
    ids = np.zeros((m, k), dtype=np.int32)
    d2 = np.zeros((m, k), dtype=np.float64)
    cnt = np.zeros(m, dtype=np.int32)
    rm = -1.0 if r_max is None else float(r_max)
    lib.or_knn(_ptr(pos), n, _ptr(centers), m, _ptr(s), _ptr(L), int(cyclic_mask), rm, int(k),
               _ptr(ids), _ptr(d2), _ptr(cnt), int(threads))
    return ids, d2, cnt


def cells_radius(pos, origin, cell_size: float, log2_cells, cyclic_mask: int, r: float, queries=None,
                 method: str = "sphere", threads: int = 0):
    """Radius lists of the points `queries` (default all; each leaves itself
    out) through a CPU cell walk of cells.c: method "sphere" (the offset
    table by minimum bound with the Eq. 1 cell test) or "cube" (the bounding
    cube of cells).  Same lists as radius(); returns (offsets, ids)."""
    lib = _load()
    pos = _f4(pos)
    n = pos.shape[0]
    q = np.arange(n, dtype=np.int64) if queries is None else np.ascontiguousarray(queries, dtype=np.int64)
    o = np.ascontiguousarray(origin, dtype=np.float64)
    w = np.ascontiguousarray(log2_cells, dtype=np.int32)
    mode = {"cube": 0, "sphere": 1}[method]
    counts = np.zeros(q.shape[0], dtype=np.int64)
    rc = lib.or_cells_radius(_ptr(pos), n, _ptr(o), float(cell_size), _ptr(w), int(cyclic_mask), float(r), mode,
                             _ptr(q), q.shape[0], _ptr(counts), None, None, int(threads))
    if rc != 0:
        raise ValueError(f"or_cells_radius failed ({rc})")
    offsets = np.zeros(q.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    ids = np.zeros(int(offsets[-1]), dtype=np.int32)
    rc = lib.or_cells_radius(_ptr(pos), n, _ptr(o), float(cell_size), _ptr(w), int(cyclic_mask), float(r), mode,
                             _ptr(q), q.shape[0], None, _ptr(offsets), _ptr(ids), int(threads))
    if rc != 0:
        raise ValueError(f"or_cells_radius failed ({rc})")
    return offsets, ids


def reduce(pos, idx, box, cyclic_mask: int, r: float, threads: int = 0):
    """Per-object energy e_i and gradient dE/dx_i (FP64) for objects idx.
    E = sum over all objects of e_i."""
    lib = _load()
    pos = _f4(pos)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    L = np.ascontiguousarray(box, dtype=np.float64)
    e = np.zeros(idx.shape[0], dtype=np.float64)
    g = np.zeros((idx.shape[0], 3), dtype=np.float64)
    lib.or_reduce(_ptr(pos), pos.shape[0], _ptr(idx), idx.shape[0], _ptr(L), int(cyclic_mask),
                  float(r), _ptr(e), _ptr(g), int(threads))
    return e, g


def reduce_all(pos, box, cyclic_mask: int, r: float, threads: int = 0):
    """reduce() for every object, through the bin lattice of or_reduce_cells
    (the same pairs and per-pair terms; only the order of each sum differs)."""
    lib = _load()
    pos = _f4(pos)
    n = pos.shape[0]
    L = np.ascontiguousarray(box, dtype=np.float64)
    e = np.zeros(n, dtype=np.float64)
    g = np.zeros((n, 3), dtype=np.float64)
    if lib.or_reduce_cells(_ptr(pos), n, _ptr(L), int(cyclic_mask), float(r), _ptr(e), _ptr(g),
                           int(threads)) != 0:
        raise MemoryError("or_reduce_cells: allocation failed")
    return e, g

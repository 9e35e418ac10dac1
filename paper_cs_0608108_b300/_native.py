"""ctypes declarations of the C ABI in include/si.h (argument marshalling only).

Loading fails loudly when libsi.so is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_PKG, "libsi.so")

SI_OK, SI_ERR_INVALID, SI_ERR_OOM, SI_ERR_CUDA, SI_ERR_CAPACITY, SI_ERR_TIMEOUT, SI_ERR_INTERNAL = range(7)
SI_METHOD_SPHERE, SI_METHOD_CUBE, SI_INCLUDE_SELF, SI_NO_SORT, SI_WALK_PAPER = 0, 1, 2, 4, 8
SI_METHOD_LIST, SI_SPHERE_ONLY, SI_WALK_PLANES, SI_NO_GROUPS, SI_FAST_D2 = 16, 32, 64, 128, 256
SI_KERNEL_POLY6_CUBED = 0

c_float3 = ctypes.c_float * 3
c_u8x3 = ctypes.c_uint8 * 3


class GridDesc(ctypes.Structure):
    _fields_ = [("origin", c_float3), ("cell_size", ctypes.c_float), ("log2_cells", c_u8x3),
                ("reserved", ctypes.c_uint8), ("cyclic_mask", ctypes.c_uint32),
                ("r_max", ctypes.c_float)]


class GridInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("d_cell_start", ctypes.c_void_p), ("d_sorted_pos", ctypes.c_void_p),
                ("d_perm", ctypes.c_void_p), ("table_entries", ctypes.c_int64),
                ("table_n_max", ctypes.c_int32), ("spec_shells", ctypes.c_int32)]


class BatchParams(ctypes.Structure):
    _fields_ = [("heavy_hits", ctypes.c_float), ("q_tile", ctypes.c_int32), ("branches", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32)]


class SceneDesc(ctypes.Structure):
    _fields_ = [("desc", GridDesc), ("d_pos", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("r", ctypes.c_float), ("d_offsets", ctypes.c_void_p), ("d_ids", ctypes.c_void_p),
                ("ids_capacity", ctypes.c_int64)]


# every exported function: name -> (restype, argtypes)
P, I64, I32, U32, F, D = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32,
                          ctypes.c_float, ctypes.c_double)
SIGNATURES = {
    "si_grid_create": (I32, [ctypes.POINTER(GridDesc), I64, ctypes.POINTER(P)]),
    "si_grid_build": (I32, [P, P, I64, P]),
    "si_build_grid": (I32, [ctypes.POINTER(GridDesc), P, I64, P, ctypes.POINTER(P)]),
    "si_grid_sync": (I32, [P, P]),
    "si_grid_get_info": (I32, [P, ctypes.POINTER(GridInfo)]),
    "si_grid_destroy": (I32, [P]),
    "si_grid_set_method": (I32, [P, F, F, F]),
    "si_query_radius": (I32, [P, P, I64, F, U32, P, P, I64, ctypes.POINTER(I64), P]),
    "si_query_radius_host": (I32, [P, P, I64, F, U32, P, P, I64, ctypes.POINTER(I64), P]),
    "si_query_knn": (I32, [P, P, I64, I32, F, U32, P, P, P, P]),
    "si_neighbor_reduce": (I32, [P, F, I32, P, P, P, P]),
    "si_neighbor_energy_noalloc": (I32, [ctypes.POINTER(GridDesc), P, I64, F, P, P]),
    "si_tune_lattice": (I32, [ctypes.POINTER(GridDesc), P, I64, P, I64, F, I32, P, I32, I32, P, P, P]),
    "si_batch_create": (I32, [ctypes.POINTER(SceneDesc), I32, U32, ctypes.POINTER(P)]),
    "si_batch_default_params": (I32, [ctypes.POINTER(BatchParams)]),
    "si_batch_create_params": (I32, [ctypes.POINTER(SceneDesc), I32, U32, ctypes.POINTER(BatchParams),
                                     ctypes.POINTER(P)]),
    "si_batch_tune": (I32, [ctypes.POINTER(SceneDesc), I32, U32, ctypes.POINTER(BatchParams), I32, I32, P, P]),
    "si_batch_run": (I32, [P, I32, P]),
    "si_batch_sync": (I32, [P, P, P]),
    "si_batch_destroy": (I32, [P]),
    "si_launch_count": (I64, []),
    "si_measure_pair_rate": (I32, [U32, ctypes.POINTER(D)]),
    "si_kernel_timing_enable": (I32, [I32]),
    "si_kernel_timing_report": (I32, [ctypes.c_char_p, ctypes.c_size_t]),
    "si_status_string": (ctypes.c_char_p, [I32]),
    "si_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """Load libsi.so (built by paper_cs_0608108_b300.build) and declare its API."""
    global _lib
    if _lib is None:
        if not os.path.exists(SO_PATH):
            raise RuntimeError(f"CUDA library {SO_PATH} is not built; run __graft_entry__.build() "
                               "or python -m paper_cs_0608108_b300.build")
        L = ctypes.CDLL(SO_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class SIError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.si_last_error().decode(errors="replace")
        super().__init__(f"{where}: {L.si_status_string(status).decode()} ({msg})")
        self.status = status


def check(status: int, where: str) -> None:
    if status != SI_OK:
        raise SIError(status, where)

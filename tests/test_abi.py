"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/si.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_cs_0608108_b300 import _native, build

HEADER = os.path.join(build.INCLUDE, "si.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(si_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.SO)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("si_build_grid", "si_query_radius", "si_query_knn", "si_neighbor_reduce",
                     "si_grid_create", "si_grid_build", "si_batch_create", "si_batch_run"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol():
    assert set(declared_functions()) == set(_native.SIGNATURES)


def test_status_strings_without_gpu(lib):
    lib.si_status_string.restype = ctypes.c_char_p
    assert lib.si_status_string(0) == b"ok"
    assert lib.si_status_string(4) == b"output capacity exceeded"


def test_descriptor_validation_needs_no_gpu(lib):
    # invalid descriptors are rejected before any device call
    L = _native.lib()
    d = _native.GridDesc()
    d.cell_size = 1.0
    d.log2_cells[0] = d.log2_cells[1] = d.log2_cells[2] = 1      # lattice axis < 4 cells
    d.cyclic_mask = 0
    d.r_max = 1.0
    h = ctypes.c_void_p()
    assert L.si_grid_create(ctypes.byref(d), 10, ctypes.byref(h)) == _native.SI_ERR_INVALID
    assert b"log2_cells" in L.si_last_error()
    d.log2_cells[0] = d.log2_cells[1] = d.log2_cells[2] = 4
    d.cyclic_mask = 7
    d.r_max = 8.0                # radius of 8 cells wraps a 16-cell cyclic axis
    assert L.si_grid_create(ctypes.byref(d), 10, ctypes.byref(h)) == _native.SI_ERR_INVALID
    d.cyclic_mask = 1
    d.r_max = float("inf")       # unbounded needs every axis non-cyclic
    assert L.si_grid_create(ctypes.byref(d), 10, ctypes.byref(h)) == _native.SI_ERR_INVALID

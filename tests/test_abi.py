"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/lpic.h declares; the header and the binding agree."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lpic.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lpic_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_13507_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_calls():
    names = declared()
    for n in ("lpic_create_grid", "lpic_add_species", "lpic_gather_push_deposit",
              "lpic_maxwell_half_step", "lpic_sort_particles"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2607_13507_b300 import lpic
    assert sorted(lpic.EXPORTS) == declared()


def test_species_bytes_layout(lib):
    f = lib.lpic_species_bytes
    f.restype = ctypes.c_size_t
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong]
    assert f(2, 1, 64) == 8 * 4 * 64        # cell, off x2, u x3, w, id
    assert f(3, 1, 128) == 9 * 4 * 128
    assert f(2, 0, 64) == 6 * 8 * 64 + 4 * 64
    assert f(3, 0, 64) == 7 * 8 * 64 + 4 * 64
    assert f(4, 1, 64) == 0


def test_descriptor_errors_are_returned_without_a_device(lib):
    """Argument checks happen on the host before any CUDA call."""
    from paper_2607_13507_b300 import lpic
    L = lpic.load()
    h = ctypes.c_void_p()
    d = lpic.GridDesc()
    d.dim = 5
    assert L.lpic_create_grid(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"dim" in L.lpic_last_error()
    d = lpic.GridDesc(2, 64, 64, 1, 0.1, 0.1, 1.0, 0.2)     # dt above the Courant limit
    assert L.lpic_create_grid(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"Courant" in L.lpic_last_error()
    d = lpic.GridDesc(2, 64, 64, 1, 0.1, 0.1, 1.0, 0.05)
    d.shape_order, d.precision, d.maxwell_fp64 = 1, lpic.FP64, 1     # FP64 master fields need FP32_FIXED
    assert L.lpic_create_grid(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"maxwell_fp64" in L.lpic_last_error()
    assert L.lpic_gather_push_deposit(None, 0, None) == 1

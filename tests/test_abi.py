"""CPU checks of the C ABI: the library builds, loads without a GPU, exports every entry point
declared in include/*.h, and rejects invalid descriptors before touching the device."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def zlib():
    from paper_2601_04826_gb300 import build, zoomy

    build.build()
    return zoomy


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(zoomy_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_core_entry_points():
    names = declared_functions()
    for n in ["zoomy_mesh_create", "zoomy_model_set", "zoomy_step", "zoomy_max_wavespeed", "zoomy_mass",
              "zoomy_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(zlib):
    L = C.CDLL(zlib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(zlib):
    bound = {n for n, _, _ in zlib._SIGNATURES}
    assert set(declared_functions()) <= bound


def test_invalid_descriptors_rejected_before_device(zlib):
    L = zlib.lib()
    h = C.c_void_p()
    assert L.zoomy_mesh_create(None, None, C.byref(h)) == zlib.ZOOMY_EINVAL
    d, _ = zlib.mesh_2d(0, 10)
    assert L.zoomy_mesh_create(C.byref(d), None, C.byref(h)) == zlib.ZOOMY_EINVAL
    assert "nx" in zlib.zoomy_last_error()
    d, _ = zlib.mesh_2d(10, 10)
    d.kind = 7
    assert L.zoomy_mesh_create(C.byref(d), None, C.byref(h)) == zlib.ZOOMY_EINVAL
    d, _ = zlib.mesh_2d(10, 10, bc=(1, 1, 2, 1))
    assert L.zoomy_mesh_create(C.byref(d), None, C.byref(h)) == zlib.ZOOMY_EINVAL
    d, _ = zlib.mesh_1d(10, 1.0, 0.0)
    assert L.zoomy_mesh_create(C.byref(d), None, C.byref(h)) == zlib.ZOOMY_EINVAL
    assert L.zoomy_model_set(None, 1, None, 9.81, 0.45, 0.0, 0) == zlib.ZOOMY_EINVAL
    assert L.zoomy_step(None, None, 0, 0.0, 1, None) == zlib.ZOOMY_EINVAL
    assert L.zoomy_mesh_destroy(None) == zlib.ZOOMY_OK
    assert zlib.zoomy_version() >= 10000

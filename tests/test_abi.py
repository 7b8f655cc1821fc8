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


def test_noalloc_rejects_bad_arguments_before_device(zlib):
    """zoomy_step_noalloc validates on the host before any CUDA call: wrapping sizes, misaligned
    pointers and negative friction coefficients are rejected with EINVAL (the pointers here are never
    dereferenced)."""
    L = zlib.lib()
    bc = (C.c_int32 * 4)(1, 1, 1, 1)
    t = C.c_double()
    Q, bed = 1 << 20, 2 << 20  # plausible aligned addresses, never touched on a rejected call

    def call(nx=64, ny=64, ld=None, fr=None, q=Q, b=bed):
        return L.zoomy_step_noalloc(nx, ny, 0.0, 1.0, 0.0, 1.0, bc, 2, C.byref(fr) if fr else None, 9.81, 0.45,
                                    1e-6, b, q, nx * ny if ld is None else ld, 0.0, 1, None, C.byref(t))

    # nx * ny beyond the 32-bit cell index (the product would wrap in the kernels)
    assert call(nx=1 << 31, ny=1, ld=1 << 31) == zlib.ZOOMY_EINVAL
    assert call(nx=1 << 16, ny=1 << 16, ld=1 << 32) == zlib.ZOOMY_EINVAL
    assert "32-bit" in zlib.zoomy_last_error()
    # misaligned float pointers
    assert call(q=Q + 2) == zlib.ZOOMY_EINVAL
    assert "aligned" in zlib.zoomy_last_error()
    assert call(b=bed + 1) == zlib.ZOOMY_EINVAL
    # friction coefficients that zoomy_model_set refuses are refused here too
    for kw in ({"C": -0.1}, {"nu": -0.01}, {"manning_n": -0.03}, {"rho": 0.0}):
        fr = zlib.friction(zlib.FRICTION_SLIP_NEWTONIAN, **kw) if "manning_n" not in kw else \
            zlib.friction(zlib.FRICTION_MANNING, **kw)
        assert call(fr=fr) == zlib.ZOOMY_EINVAL, kw
        assert "friction" in zlib.zoomy_last_error()
    # ld below the cell count
    assert call(ld=64 * 64 - 1) == zlib.ZOOMY_EINVAL

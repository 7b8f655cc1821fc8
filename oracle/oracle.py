"""FP64 CPU oracle of the shallow-moment finite-volume step -- TEST INFRASTRUCTURE ONLY.

Python side of ``zoomy_oracle.c`` (the scheme itself) and the FP64 MLP of the
learned closure (``mlp_*``).  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the library in
``paper_2601_04826_gb300`` never does, and this module imports nothing from it.

The C part is compiled with gcc (``-O2 -ffp-contract=off``, OpenMP over cells
when available) into ``oracle/_build/``.  Every function here only marshals
numpy arrays; the arithmetic is in the C file or written out below in numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "zoomy_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libzoomy_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP64, no FMA contraction). Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    """The compiled oracle; ZOOMY_ORACLE_LIB may name another build of the same source
    (the mutation tests use this to load deliberately broken copies)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("ZOOMY_ORACLE_LIB") or build()
            _lib = C.CDLL(path)
            _declare(_lib)
    return _lib


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_ip32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def _declare(L):
    vp = C.c_void_p
    L.or_basis_tables.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp]
    L.or_model_new.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double,
                               C.c_double, C.c_double, C.c_double]
    L.or_model_new.restype = vp
    L.or_model_free.argtypes = [vp]
    L.or_model_set_source_mode.argtypes = [vp, C.c_int]
    L.or_model_set_order.argtypes = [vp, C.c_int]
    L.or_friction_implicit.argtypes = [vp, _dp, C.c_double]
    L.or_model_nv.argtypes = [vp]
    L.or_flux.argtypes = [vp, _dp, C.c_double, C.c_double, _dp]
    L.or_nc_matrix.argtypes = [vp, _dp, C.c_double, C.c_double, _dp]
    L.or_wavespeed.argtypes = [vp, _dp]
    L.or_wavespeed.restype = C.c_double
    L.or_source_newtonian.argtypes = [vp, _dp, _dp]
    L.or_bottom_friction.argtypes = [vp, _dp, C.c_double]
    L.or_mesh_1d.argtypes = [C.c_int64, C.c_double, C.c_double, C.c_int, C.c_int]
    L.or_mesh_1d.restype = vp
    L.or_mesh_2d.argtypes = [C.c_int64, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double,
                             _ip32]
    L.or_mesh_2d.restype = vp
    L.or_mesh_tri.argtypes = [C.c_int64, _dp, C.c_int64, _ip32, C.c_int]
    L.or_mesh_tri.restype = vp
    L.or_lift3d.argtypes = [vp, vp, _dp, vp, C.c_int, _dp, _dp]
    L.or_mesh_free.argtypes = [vp]
    L.or_mesh_ncells.argtypes = [vp]
    L.or_mesh_ncells.restype = C.c_int64
    L.or_mesh_geometry.argtypes = [vp, _dp, _dp, _ip64, _dp, _dp, _dp]
    L.or_stage.argtypes = [vp, vp, _dp, vp, C.c_double, _dp]
    L.or_step.argtypes = [vp, vp, _dp, vp, C.c_double, C.c_double, C.c_int,
                          C.POINTER(C.c_double)]
    L.or_step_ex.argtypes = [vp, vp, _dp, vp, C.c_double, C.c_double, C.c_int, C.c_int,
                             C.POINTER(C.c_double)]
    L.or_max_wavespeed.argtypes = [vp, vp, _dp]
    L.or_max_wavespeed.restype = C.c_double
    L.or_min_delta.argtypes = [vp]
    L.or_min_delta.restype = C.c_double
    L.or_cfl_dt.argtypes = [vp, vp, _dp, C.c_double]
    L.or_cfl_dt.restype = C.c_double
    L.or_mass.argtypes = [vp, _dp]
    L.or_mass.restype = C.c_double
    L.or_max_level.restype = C.c_int
    L.or_closure_new.argtypes = [_dp, _dp, _dp, C.c_int]
    L.or_closure_new.restype = vp
    L.or_closure_free.argtypes = [vp]
    L.or_closure_eval.argtypes = [vp, _dp, _dp]
    L.or_closure_max_wavespeed.argtypes = [vp, vp, vp, _dp]
    L.or_closure_max_wavespeed.restype = C.c_double
    L.or_step_closure.argtypes = [vp, vp, vp, _dp, vp, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                                  C.POINTER(C.c_double)]


# --------------------------------------------------------------------------- basis

def basis_tables(N: int):
    """Basis integrals M[k], A[i,j,k], B[k,j,l], C[i,k], phi_k(0) of the shifted Legendre basis."""
    m = N + 1
    M = np.zeros(m)
    A = np.zeros(m * m * m)
    B = np.zeros(m * m * m)
    Cm = np.zeros(m * m)
    p0 = np.zeros(m)
    if lib().or_basis_tables(N, M, A, B, Cm, p0) != 0:
        raise ValueError("level out of range")
    return M, A.reshape(m, m, m), B.reshape(m, m, m), Cm.reshape(m, m), p0


# --------------------------------------------------------------------------- model

FRICTION_NONE, FRICTION_SLIP_NEWTONIAN, FRICTION_MANNING = 0, 1, 2


class Model:
    """Level-N shallow-moment model in 1D or 2D (variable order documented in the C file)."""

    def __init__(self, N, dim, g=9.81, h_dry=1e-6, friction=0, C=0.0, nu=0.0, rho=1.0, manning_n=0.0,
                 implicit_source=False, order=1):
        self.N, self.dim = N, dim
        self._p = lib().or_model_new(N, dim, g, h_dry, friction, C, nu, rho, manning_n)
        if not self._p:
            raise ValueError("bad model parameters")
        # reading R17: friction (Newtonian + bottom stress) by backward Euler after each stage
        lib().or_model_set_source_mode(self._p, 1 if implicit_source else 0)
        # reading R18: order 2 = MUSCL reconstruction on 1D and structured 2D meshes
        if order not in (1, 2):
            raise ValueError("order is 1 or 2")
        lib().or_model_set_order(self._p, order)
        self.nv = lib().or_model_nv(self._p)
        self.g, self.h_dry = g, h_dry

    def __del__(self):
        if getattr(self, "_p", None):
            lib().or_model_free(self._p)
            self._p = None

    def flux(self, q, nx=1.0, ny=0.0):
        F = np.zeros(self.nv)
        lib().or_flux(self._p, np.ascontiguousarray(q, dtype=np.float64), nx, ny, F)
        return F

    def nc_matrix(self, q, nx=1.0, ny=0.0):
        Bn = np.zeros(self.nv * self.nv)
        lib().or_nc_matrix(self._p, np.ascontiguousarray(q, dtype=np.float64), nx, ny, Bn)
        return Bn.reshape(self.nv, self.nv)

    def wavespeed(self, q):
        return lib().or_wavespeed(self._p, np.ascontiguousarray(q, dtype=np.float64))

    def source_newtonian(self, q):
        S = np.zeros(self.nv)
        lib().or_source_newtonian(self._p, np.ascontiguousarray(q, dtype=np.float64), S)
        return S

    def bottom_friction(self, y, dt):
        y = np.array(y, dtype=np.float64)
        lib().or_bottom_friction(self._p, y, dt)
        return y

    def friction_implicit(self, y, dt):
        y = np.array(y, dtype=np.float64)
        lib().or_friction_implicit(self._p, y, dt)
        return y

    def index_alpha(self, k):
        return 1 + k if self.dim == 1 else (1 if k == 0 else 2 + k)

    def index_beta(self, k):
        return 2 if k == 0 else 2 + self.N + k


# --------------------------------------------------------------------------- mesh

class Mesh:
    def __init__(self, ptr, nf):
        self._p = ptr
        self.nf = nf
        self.nc = lib().or_mesh_ncells(ptr)

    def __del__(self):
        if getattr(self, "_p", None):
            lib().or_mesh_free(self._p)
            self._p = None

    @staticmethod
    def line(nx, x0, x1, bc_left=0, bc_right=0):
        return Mesh(lib().or_mesh_1d(nx, x0, x1, bc_left, bc_right), 2)

    @staticmethod
    def rect(nx, ny, x0, x1, y0, y1, bc=(0, 0, 0, 0)):
        return Mesh(lib().or_mesh_2d(nx, ny, x0, x1, y0, y1, np.asarray(bc, dtype=np.int32)), 4)

    @staticmethod
    def triangles(verts_xy, tris, bc=1):
        v = np.ascontiguousarray(verts_xy, dtype=np.float64).reshape(-1)
        t = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1)
        return Mesh(lib().or_mesh_tri(len(v) // 2, v, len(t) // 3, t, bc), 3)

    def geometry(self):
        nc, nf = self.nc, self.nf
        area, delta = np.zeros(nc), np.zeros(nc)
        nbr = np.zeros(nc * nf, dtype=np.int64)
        fnx, fny, flen = np.zeros(nc * nf), np.zeros(nc * nf), np.zeros(nc * nf)
        lib().or_mesh_geometry(self._p, area, delta, nbr, fnx, fny, flen)
        return dict(area=area, delta=delta, nbr=nbr.reshape(nc, nf), nx=fnx.reshape(nc, nf),
                    ny=fny.reshape(nc, nf), len=flen.reshape(nc, nf))

    def min_delta(self):
        return lib().or_min_delta(self._p)


def _bed_ptr(bed):
    if bed is None:
        return None, None
    b = np.ascontiguousarray(bed, dtype=np.float64)
    return b, b.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------- scheme

def stage(model, mesh, X, dt, bed=None):
    """One explicit stage Y = R(X + dt L(X)); X is [nv, ncells] float64."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.zeros_like(X)
    b, bp = _bed_ptr(bed)
    lib().or_stage(model._p, mesh._p, X, bp, dt, Y)
    return Y


def step(model, mesh, Q, nsteps, dt=0.0, cfl=0.45, bed=None, store_f32=False):
    """nsteps SSP-RK2 steps (dt > 0 fixed, dt <= 0 adaptive CFL). Returns (Q_new, t_advanced).

    store_f32 keeps the state in single precision between stages (FP64 arithmetic on it), the
    precision form of an FP32-state implementation."""
    Q = np.array(Q, dtype=np.float64, order="C")
    b, bp = _bed_ptr(bed)
    t = C.c_double(0.0)
    lib().or_step_ex(model._p, mesh._p, Q, bp, dt, cfl, nsteps, 1 if store_f32 else 0, C.byref(t))
    return Q, t.value


def max_wavespeed(model, mesh, Q):
    return lib().or_max_wavespeed(model._p, mesh._p, np.ascontiguousarray(Q, dtype=np.float64))


def cfl_dt(model, mesh, Q, cfl):
    return lib().or_cfl_dt(model._p, mesh._p, np.ascontiguousarray(Q, dtype=np.float64), cfl)


def mass(mesh, Q):
    return lib().or_mass(mesh._p, np.ascontiguousarray(Q, dtype=np.float64))


def lift3d(model, mesh, Q, zeta, bed=None):
    """Three-dimensional fields at sigma levels zeta (Sec. "Postprocessing", interpolate_3d):
    returns [4, K, nc] = u, v, w, p (see or_lift3d)."""
    Qc = np.ascontiguousarray(Q, dtype=np.float64)
    z = np.ascontiguousarray(zeta, dtype=np.float64)
    out = np.zeros((4, len(z), Qc.shape[1]))
    b, bp = _bed_ptr(bed)
    lib().or_lift3d(model._p, mesh._p, Qc, bp, len(z), z, out)
    return out


def max_level():
    return lib().or_max_level()


# --------------------------------------------------------------------------- learned closure

class Closure:
    """The closure MLP in the C oracle (params in the order of mlp.pack, FP64; bf16 mirrors the
    inference kernel's BF16 layer inputs)."""

    def __init__(self, params, in_scale, out_scale, bf16=True):
        self._p = lib().or_closure_new(np.ascontiguousarray(params, dtype=np.float64),
                                       np.ascontiguousarray(in_scale, dtype=np.float64),
                                       np.ascontiguousarray(out_scale, dtype=np.float64), 1 if bf16 else 0)

    def __del__(self):
        if getattr(self, "_p", None):
            lib().or_closure_free(self._p)
            self._p = None

    def eval(self, feat):
        out = np.zeros(6)
        lib().or_closure_eval(self._p, np.ascontiguousarray(feat, dtype=np.float64), out)
        return out


def step_closure(model4, closure, mesh, Q1, nsteps, dt=0.0, cfl=0.45, bed=None, store_f32=False, schedule=0):
    """nsteps SSP-RK2 steps of the closure model (level-1 state [5, nc], level-4 model); schedule 0
    evaluates the network on every stage input, 1 once per step on Q^n (held for both stages)."""
    Q = np.array(Q1, dtype=np.float64, order="C")
    b, bp = _bed_ptr(bed)
    t = C.c_double(0.0)
    rc = lib().or_step_closure(model4._p, closure._p, mesh._p, Q, bp, dt, cfl, nsteps, 1 if store_f32 else 0,
                               int(schedule), C.byref(t))
    if rc != 0:
        raise ValueError("closure step needs a 2D level-4 model")
    return Q, t.value


def closure_max_wavespeed(model4, closure, mesh, Q1):
    return lib().or_closure_max_wavespeed(model4._p, closure._p, mesh._p, np.ascontiguousarray(Q1, dtype=np.float64))

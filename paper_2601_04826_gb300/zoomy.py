"""Thin ctypes binding of the C ABI in include/zoomy.h (argument marshalling only).

Every function keeps the C name and argument order.  Device buffers are passed
as torch CUDA tensors (their ``data_ptr()``) or raw integers; the stream is the
current torch stream unless one is given.  Nothing here computes any part of
the method: all of it runs in libzoomy.so, and a missing library raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# ZOOMY_LIBRARY may name another build of the same sources (the bounds-checking libzoomy_debug.so)
LIB_PATH = os.environ.get("ZOOMY_LIBRARY") or os.path.join(HERE, "libzoomy.so")

(ZOOMY_OK, ZOOMY_EINVAL, ZOOMY_ENOMEM, ZOOMY_ECUDA, ZOOMY_ENAN, ZOOMY_ENEGDEPTH, ZOOMY_ECFL, ZOOMY_ETIMEOUT, ZOOMY_ESTATE,
 ZOOMY_EBOUNDS) = range(10)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENAN", "ENEGDEPTH", "ECFL", "ETIMEOUT", "ESTATE", "EBOUNDS"]
MESH_1D, MESH_2D, MESH_TRI = 0, 1, 2
BC_TRANSMISSIVE, BC_WALL = 0, 1
FRICTION_NONE, FRICTION_SLIP_NEWTONIAN, FRICTION_MANNING = 0, 1, 2
FP32, FP64 = 0, 1
LAUNCH_AUTO, LAUNCH_PER_STAGE, LAUNCH_PERSISTENT = 0, 1, 2


class ZoomyError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class zoomy_mesh_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nx", C.c_int64), ("ny", C.c_int64), ("x0", C.c_double), ("x1", C.c_double),
                ("y0", C.c_double), ("y1", C.c_double), ("bc", C.c_int32 * 4), ("nverts", C.c_int64),
                ("ntris", C.c_int64), ("verts_xy", C.c_void_p), ("tris", C.c_void_p), ("bathymetry", C.c_void_p),
                ("morton_reorder", C.c_int32)]


class zoomy_friction(C.Structure):
    _fields_ = [("kind", C.c_int32), ("C", C.c_double), ("nu", C.c_double), ("rho", C.c_double),
                ("manning_n", C.c_double)]


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes) for every entry point of include/zoomy.h
_SIGNATURES = [
    ("zoomy_version", C.c_int32, []),
    ("zoomy_mesh_create", C.c_int, [C.POINTER(zoomy_mesh_desc), C.c_void_p, C.POINTER(C.c_void_p)]),
    ("zoomy_mesh_destroy", C.c_int, [C.c_void_p]),
    ("zoomy_set_stream", C.c_int, [C.c_void_p, C.c_void_p]),
    ("zoomy_mesh_info", C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    ("zoomy_mesh_permutation", C.c_int, [C.c_void_p, C.c_void_p]),
    ("zoomy_model_set", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(zoomy_friction), C.c_double, C.c_double,
                                  C.c_double, C.c_int32]),
    ("zoomy_nvars", C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    ("zoomy_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_int32, C.POINTER(C.c_double)]),
    ("zoomy_step_host", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_int32,
                                  C.POINTER(C.c_double)]),
    ("zoomy_sync", C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    ("zoomy_max_wavespeed", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double)]),
    ("zoomy_mass", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double)]),
    ("zoomy_tune_set", C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    ("zoomy_tune_1d", C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    ("zoomy_autotune", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_char_p, C.POINTER(C.c_int32),
                                 C.POINTER(C.c_double)]),
    ("zoomy_closure_set", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double]),
    ("zoomy_closure_clear", C.c_int, [C.c_void_p]),
    ("zoomy_closure_eval", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    ("zoomy_closure_engine", C.c_int, [C.c_void_p, C.c_int32]),
    ("zoomy_source_mode", C.c_int, [C.c_void_p, C.c_int32]),
    ("zoomy_space_order", C.c_int, [C.c_void_p, C.c_int32]),
    ("zoomy_vam_set", C.c_int, [C.c_void_p, C.c_int32]),
    ("zoomy_lift3d", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_int64]),
    ("zoomy_mlp_create", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("zoomy_mlp_destroy", C.c_int, [C.c_void_p]),
    ("zoomy_mlp_get_params", C.c_int, [C.c_void_p, C.c_void_p]),
    ("zoomy_mlp_grad", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_float),
                                 C.c_void_p]),
    ("zoomy_mlp_train_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float,
                                       C.POINTER(C.c_float)]),
    ("zoomy_closure_samples", C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_double,
                                        C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("zoomy_ensemble_create", C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_double,
                                        C.c_double, C.c_double, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("zoomy_ensemble_offsets", C.c_int, [C.c_void_p, C.c_void_p]),
    ("zoomy_ensemble_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p]),
    ("zoomy_ensemble_autotune", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int32),
                                          C.POINTER(C.c_double)]),
    ("zoomy_ensemble_set_barrier", C.c_int, [C.c_void_p, C.c_int64, C.c_int32]),
    ("zoomy_profile_enable", C.c_int, [C.c_void_p, C.c_int32]),
    ("zoomy_profile_read", C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    ("zoomy_closure_schedule", C.c_int, [C.c_void_p, C.c_int32]),
    ("zoomy_advance", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_int32, C.POINTER(C.c_double),
                                C.POINTER(C.c_int64)]),
    ("zoomy_sample_scales", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_float),
                                      C.POINTER(C.c_float), C.c_void_p]),
    ("zoomy_sample_scale", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("zoomy_step_noalloc", C.c_int, [C.c_int64, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double,
                                     C.POINTER(C.c_int32), C.c_int32, C.POINTER(zoomy_friction), C.c_double,
                                     C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_int64, C.c_double,
                                     C.c_int32, C.c_void_p, C.POINTER(C.c_double)]),
    ("zoomy_last_error", C.c_char_p, []),
]


def lib():
    """Open libzoomy.so (raises if it has not been built; there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise OSError(f"{LIB_PATH} is missing: build it with paper_2601_04826_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            for name, res, args in _SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(st):
    if st != ZOOMY_OK:
        raise ZoomyError(st, lib().zoomy_last_error().decode())
    return st


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ----------------------------------------------------------------------------- C entry points

def zoomy_version():
    return lib().zoomy_version()


def zoomy_mesh_create(desc: zoomy_mesh_desc, stream=None):
    h = C.c_void_p()
    _check(lib().zoomy_mesh_create(C.byref(desc), _stream(stream), C.byref(h)))
    return h.value


def zoomy_mesh_destroy(ctx):
    _check(lib().zoomy_mesh_destroy(ctx))


def zoomy_set_stream(ctx, stream=None):
    _check(lib().zoomy_set_stream(ctx, _stream(stream)))


def zoomy_mesh_info(ctx):
    n = C.c_int64()
    d = C.c_double()
    _check(lib().zoomy_mesh_info(ctx, C.byref(n), C.byref(d)))
    return n.value, d.value


def zoomy_mesh_permutation(ctx, perm_out):
    _check(lib().zoomy_mesh_permutation(ctx, _ptr(perm_out)))
    return perm_out


def zoomy_model_set(ctx, level, friction: zoomy_friction | None, g=9.81, cfl=0.45, h_dry=1e-6, dtype=FP32):
    _check(lib().zoomy_model_set(ctx, level, C.byref(friction) if friction is not None else None, g, cfl, h_dry,
                                 dtype))


def zoomy_nvars(ctx):
    nv = C.c_int32()
    _check(lib().zoomy_nvars(ctx, C.byref(nv)))
    return nv.value


def zoomy_step(ctx, Q, ld, dt, nsteps, sync=True):
    t = C.c_double()
    _check(lib().zoomy_step(ctx, _ptr(Q), ld, dt, nsteps, C.byref(t) if sync else None))
    return t.value if sync else None


def zoomy_step_host(ctx, Q_host, ld, dt, nsteps):
    t = C.c_double()
    _check(lib().zoomy_step_host(ctx, _ptr(Q_host), ld, dt, nsteps, C.byref(t)))
    return t.value


def zoomy_sync(ctx):
    t = C.c_double()
    _check(lib().zoomy_sync(ctx, C.byref(t)))
    return t.value


def zoomy_max_wavespeed(ctx, Q, ld):
    out = C.c_double()
    _check(lib().zoomy_max_wavespeed(ctx, _ptr(Q), ld, C.byref(out)))
    return out.value


def zoomy_mass(ctx, Q, ld):
    out = C.c_double()
    _check(lib().zoomy_mass(ctx, _ptr(Q), ld, C.byref(out)))
    return out.value


def zoomy_tune_set(ctx, rows_per_warp, warps_per_block):
    _check(lib().zoomy_tune_set(ctx, rows_per_warp, warps_per_block))


def zoomy_tune_1d(ctx, mode, warps_per_cta=0):
    _check(lib().zoomy_tune_1d(ctx, mode, warps_per_cta))


def zoomy_autotune(ctx, Q, ld, cache_path=None):
    h = C.c_int32()
    us = C.c_double()
    _check(lib().zoomy_autotune(ctx, _ptr(Q), ld, cache_path.encode() if cache_path else None, C.byref(h),
                                C.byref(us)))
    return h.value, us.value


def zoomy_closure_set(ctx, params, in_scale, out_scale, lam):
    import numpy as np

    p = np.ascontiguousarray(params, dtype=np.float32)
    i = np.ascontiguousarray(in_scale, dtype=np.float32)
    o = np.ascontiguousarray(out_scale, dtype=np.float32)
    _check(lib().zoomy_closure_set(ctx, p.ctypes.data, i.ctypes.data, o.ctypes.data, lam))


def zoomy_closure_clear(ctx):
    _check(lib().zoomy_closure_clear(ctx))


def zoomy_closure_eval(ctx, feat, out, n):
    _check(lib().zoomy_closure_eval(ctx, _ptr(feat), _ptr(out), n))


def zoomy_closure_engine(ctx, engine):
    _check(lib().zoomy_closure_engine(ctx, engine))


def zoomy_source_mode(ctx, mode):
    _check(lib().zoomy_source_mode(ctx, mode))


def zoomy_space_order(ctx, order):
    _check(lib().zoomy_space_order(ctx, order))


def zoomy_vam_set(ctx, enable=1):
    _check(lib().zoomy_vam_set(ctx, enable))


def zoomy_lift3d(ctx, Q, ld, zeta, out, ldo):
    import numpy as np

    z = np.ascontiguousarray(zeta, dtype=np.float64)
    _check(lib().zoomy_lift3d(ctx, _ptr(Q), ld, len(z), z.ctypes.data, _ptr(out), ldo))


def zoomy_mlp_create(params, stream=None):
    import numpy as np

    p = np.ascontiguousarray(params, dtype=np.float32)
    h = C.c_void_p()
    _check(lib().zoomy_mlp_create(p.ctypes.data, _stream(stream), C.byref(h)))
    return h.value


def zoomy_mlp_destroy(mlp):
    _check(lib().zoomy_mlp_destroy(mlp))


def zoomy_mlp_get_params(mlp):
    import numpy as np

    p = np.zeros(4998, dtype=np.float32)
    _check(lib().zoomy_mlp_get_params(mlp, p.ctypes.data))
    return p


def zoomy_mlp_grad(mlp, X, T, n):
    import numpy as np

    loss = C.c_float()
    g = np.zeros(4998, dtype=np.float32)
    _check(lib().zoomy_mlp_grad(mlp, _ptr(X), _ptr(T), n, C.byref(loss), g.ctypes.data))
    return loss.value, g


def zoomy_mlp_train_step(mlp, X, T, n, lr, want_loss=False):
    loss = C.c_float()
    _check(lib().zoomy_mlp_train_step(mlp, _ptr(X), _ptr(T), n, lr, C.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def zoomy_closure_samples(Q, ld, level, cells, n, lam, h_dry, in_scale, out_scale, X, T, stream=None):
    _check(lib().zoomy_closure_samples(_ptr(Q), ld, level, _ptr(cells), n, lam, h_dry, _ptr(in_scale),
                                       _ptr(out_scale), _ptr(X), _ptr(T), _stream(stream)))


def zoomy_ensemble_create(sides, slip, level, nu=0.01, g=9.81, cfl=0.45, h_dry=1e-6, stream=None):
    import numpy as np

    sd = np.ascontiguousarray(sides, dtype=np.int64)
    cc = np.ascontiguousarray(slip, dtype=np.float64)
    h = C.c_void_p()
    _check(lib().zoomy_ensemble_create(len(sd), sd.ctypes.data, cc.ctypes.data, level, nu, g, cfl, h_dry,
                                       _stream(stream), C.byref(h)))
    return h.value


def zoomy_ensemble_offsets(ctx, nmembers):
    import numpy as np

    off = np.zeros(nmembers + 1, dtype=np.int64)
    _check(lib().zoomy_ensemble_offsets(ctx, off.ctypes.data))
    return off


def zoomy_ensemble_step(ctx, Q, ld, nsteps, mode=0, nmembers=None):
    import numpy as np

    t = np.zeros(nmembers, dtype=np.float64) if nmembers else None
    _check(lib().zoomy_ensemble_step(ctx, _ptr(Q), ld, nsteps, mode, t.ctypes.data if t is not None else None))
    return t


def zoomy_ensemble_autotune(ctx, Q, ld):
    h = C.c_int32()
    us = C.c_double()
    _check(lib().zoomy_ensemble_autotune(ctx, _ptr(Q), ld, C.byref(h), C.byref(us)))
    return h.value, us.value


def zoomy_ensemble_set_barrier(ctx, spin_limit=20000000, extra_participants=0):
    _check(lib().zoomy_ensemble_set_barrier(ctx, spin_limit, extra_participants))


def zoomy_profile_enable(ctx, on=True):
    _check(lib().zoomy_profile_enable(ctx, 1 if on else 0))


def zoomy_profile_read(ctx):
    n = (C.c_int64 * 3)()
    ms = (C.c_double * 3)()
    _check(lib().zoomy_profile_read(ctx, n, ms))
    return list(n), list(ms)


def zoomy_step_noalloc(nx, ny, x0, x1, y0, y1, bc, level, friction, g, cfl, h_dry, bed, Q, ld, dt, nsteps,
                       stream=None, sync=True):
    """The allocation-free step (see include/zoomy.h): every argument is passed through unchanged."""
    bcs = (C.c_int32 * 4)(*bc)
    t = C.c_double()
    _check(lib().zoomy_step_noalloc(nx, ny, x0, x1, y0, y1, bcs, level,
                                    C.byref(friction) if friction is not None else None, g, cfl, h_dry, _ptr(bed),
                                    _ptr(Q), ld, dt, nsteps, _stream(stream), C.byref(t) if sync else None))
    return t.value if sync else None


def zoomy_advance(ctx, Q, ld, t_end, chunk=256):
    t = C.c_double()
    n = C.c_int64()
    _check(lib().zoomy_advance(ctx, _ptr(Q), ld, t_end, chunk, C.byref(t), C.byref(n)))
    return t.value, n.value


def zoomy_sample_scales(X, T, n, stream=None):
    ins = (C.c_float * 6)()
    outs = (C.c_float * 6)()
    _check(lib().zoomy_sample_scales(_ptr(X), _ptr(T), n, ins, outs, _stream(stream)))
    return list(ins), list(outs)


def zoomy_sample_scale(X, T, n, in_scale, out_scale, stream=None):
    _check(lib().zoomy_sample_scale(_ptr(X), _ptr(T), n, _ptr(in_scale), _ptr(out_scale), _stream(stream)))


def zoomy_closure_schedule(ctx, schedule):
    _check(lib().zoomy_closure_schedule(ctx, schedule))


def zoomy_last_error():
    return lib().zoomy_last_error().decode()


# ----------------------------------------------------------------------------- descriptors

def mesh_1d(nx, x0, x1, bc=(0, 0), bathymetry=None):
    d = zoomy_mesh_desc()
    d.kind, d.nx, d.ny, d.x0, d.x1 = MESH_1D, nx, 1, x0, x1
    d.bc[0], d.bc[1] = bc
    keep = _bathy(d, bathymetry)
    return d, keep


def mesh_2d(nx, ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc=(1, 1, 1, 1), bathymetry=None):
    d = zoomy_mesh_desc()
    d.kind, d.nx, d.ny, d.x0, d.x1, d.y0, d.y1 = MESH_2D, nx, ny, x0, x1, y0, y1
    for i in range(4):
        d.bc[i] = bc[i]
    keep = _bathy(d, bathymetry)
    return d, keep


def mesh_tri(verts_xy, tris, bc=1, bathymetry=None, morton=True):
    import numpy as np

    v = np.ascontiguousarray(verts_xy, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    d = zoomy_mesh_desc()
    d.kind, d.nverts, d.ntris = MESH_TRI, len(v), len(t)
    d.verts_xy, d.tris = v.ctypes.data, t.ctypes.data
    d.bc[0] = bc
    d.morton_reorder = 1 if morton else 0
    keep = [v, t] + _bathy(d, bathymetry)
    return d, keep


def _bathy(d, bathymetry):
    if bathymetry is None:
        d.bathymetry = None
        return []
    import numpy as np

    b = np.ascontiguousarray(bathymetry, dtype=np.float64)
    d.bathymetry = b.ctypes.data
    return [b]


def friction(kind=FRICTION_NONE, C=0.0, nu=0.0, rho=1.0, manning_n=0.0):
    f = zoomy_friction()
    f.kind, f.C, f.nu, f.rho, f.manning_n = kind, C, nu, rho, manning_n
    return f


class Context:
    """Owns one zoomy_ctx; ``step`` marshals a torch CUDA tensor of shape [nv, ld]."""

    def __init__(self, desc_and_keep, level, fric=None, g=9.81, cfl=0.45, h_dry=1e-6, dtype=FP32, stream=None):
        desc, keep = desc_and_keep
        self.ctx = zoomy_mesh_create(desc, stream)
        self.ncells, self.min_delta = zoomy_mesh_info(self.ctx)
        zoomy_model_set(self.ctx, level, fric, g, cfl, h_dry, dtype)
        self.nv = zoomy_nvars(self.ctx)
        self.dtype = dtype

    def close(self):
        if getattr(self, "ctx", None):
            zoomy_mesh_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ld(self, Q):
        assert Q.dim() == 2 and Q.shape[0] == self.nv and Q.stride(1) == 1 and Q.is_cuda
        return Q.stride(0)

    def step(self, Q, nsteps=1, dt=0.0, sync=True):
        return zoomy_step(self.ctx, Q, self._ld(Q), dt, nsteps, sync)

    def step_host(self, Q_host, nsteps=1, dt=0.0):
        return zoomy_step_host(self.ctx, Q_host, Q_host.stride(0), dt, nsteps)

    def advance(self, Q, t_end, chunk=256):
        """CFL steps to t_end exactly (zoomy_advance): returns (time advanced, steps)."""
        return zoomy_advance(self.ctx, Q, self._ld(Q), t_end, chunk)

    def max_wavespeed(self, Q):
        return zoomy_max_wavespeed(self.ctx, Q, self._ld(Q))

    def mass(self, Q):
        return zoomy_mass(self.ctx, Q, self._ld(Q))

    def vam(self, enable=True):
        """Switch a 1D FP64 context to the VAM model (or back); the state then has zoomy_nvars rows."""
        zoomy_vam_set(self.ctx, 1 if enable else 0)
        self.nv = zoomy_nvars(self.ctx)

    def tune(self, rows_per_warp, warps_per_block):
        zoomy_tune_set(self.ctx, rows_per_warp, warps_per_block)

    def tune_1d(self, mode, warps_per_cta=0):
        """Launch shape of a first-order 1D line (LAUNCH_AUTO / LAUNCH_PER_STAGE / LAUNCH_PERSISTENT)."""
        zoomy_tune_1d(self.ctx, mode, warps_per_cta)

    def autotune(self, Q, cache_path=None):
        return zoomy_autotune(self.ctx, Q, self._ld(Q), cache_path)

    def permutation(self):
        import numpy as np

        p = np.zeros(self.ncells, dtype=np.int64)
        zoomy_mesh_permutation(self.ctx, p)
        return p

"""Precision report of the GPU paths against the FP64 oracle: relative L1 error per variable after the
run, for the FP64 path and for the FP32-state path (FP32 state, FP64-grade hydrostatic differences),
on one case of each workload family.  The FP32 path is compared with the plain FP64 oracle and with
the oracle's FP32-state form (the state rounded to float between stages); the bars are the parity
bars (FP64 1e-12, FP32 1e-5 against the form that shares its state rounding).  Run with -s to print
the table."""
import numpy as np
import pytest

from gpu_util import rel_l1, rounded, to_device
from paper_2601_04826_gb300 import inputs

pytestmark = pytest.mark.gpu
G = 9.81


@pytest.fixture(scope="module")
def Z():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04826_gb300 import build, zoomy

    build.build()
    return zoomy


def gpu_run(Z, desc, level, fric, Q0, nsteps, dtype, perm=None):
    kind, C_, nu, mn = fric
    ctx = Z.Context(desc, level, Z.friction(kind, C=C_, nu=nu, manning_n=mn), g=G, cfl=0.45, dtype=dtype)
    if perm is None and desc[0].kind == 2:
        perm = ctx.permutation()
    Q = to_device(Q0 if perm is None else Q0[:, perm], dtype)
    ctx.step(Q, nsteps=nsteps, dt=0.0)
    out = Q.double().cpu().numpy()
    ctx.close()
    if perm is None:
        return out
    got = np.empty_like(out)
    got[:, perm] = out
    return got


def oracle_run(oracle, mesh, level, dim, fric, Q0, nsteps, bed, store_f32=False):
    kind, C_, nu, mn = fric
    md = oracle.Model(level, dim, g=G, h_dry=1e-6, friction=kind, C=C_, nu=nu, manning_n=mn)
    ref, _ = oracle.step(md, mesh, Q0, nsteps, cfl=0.45, bed=bed, store_f32=store_f32)
    return ref


def fmt(err):
    return f"{np.max(err):.1e} (h {err[0]:.1e})"


def test_precision_table(Z, oracle):
    rows, fails = [], []

    def record(case, dtype, err64, err32form, bar_err, bar):
        rows.append((case, "FP64" if dtype == 1 else "FP32", fmt(err64), "-" if err32form is None else fmt(err32form),
                     f"{bar:.0e}"))
        if not np.all(bar_err <= bar):
            fails.append((case, dtype, bar_err))

    # config-1 family: 1D level-1 dam break, 2000 cells, 200 CFL steps, slip 0.1 + Newtonian 0.01
    fr = (1, 0.1, 0.01, 0.0)
    Q0 = inputs.dambreak_1d(2000, 0.0, 10.0, 2.0, 1.0, 5.0, level=1)
    mesh = oracle.Mesh.line(2000, 0.0, 10.0, 0, 0)
    for dt_ in (1, 0):
        Qr = rounded(Q0, dt_)
        got = gpu_run(Z, Z.mesh_1d(2000, 0.0, 10.0, bc=(0, 0)), 1, fr, Qr, 200, dt_)
        e64 = rel_l1(got, oracle_run(oracle, mesh, 1, 1, fr, Qr, 200, None))
        e32 = None if dt_ == 1 else rel_l1(got, oracle_run(oracle, mesh, 1, 1, fr, Qr, 200, None, store_f32=True))
        record("1D dam break, level 1, 2000 cells, 200 steps", dt_, e64, e32, e64 if dt_ == 1 else e32,
               1e-12 if dt_ == 1 else 1e-5)

    # config-2 family: the bench's recipe (Gaussian bump over 8-mode Fourier bathymetry) at 256^2,
    # level 2, walls, 20 steps
    Q0, b = inputs.gaussian_bump_2d(256, 256, 2, seed=0)
    mesh = oracle.Mesh.rect(256, 256, 0, 1, 0, 1, bc=(1, 1, 1, 1))
    for dt_ in (1, 0):
        Qr, br = rounded(Q0, dt_), rounded(b, dt_)
        got = gpu_run(Z, Z.mesh_2d(256, 256, bathymetry=br), 2, fr, Qr, 20, dt_)
        e64 = rel_l1(got, oracle_run(oracle, mesh, 2, 2, fr, Qr, 20, br))
        e32 = None if dt_ == 1 else rel_l1(got, oracle_run(oracle, mesh, 2, 2, fr, Qr, 20, br, store_f32=True))
        record("2D level 2, 256^2, bathymetry, walls, 20 steps", dt_, e64, e32, e64 if dt_ == 1 else e32,
               1e-12 if dt_ == 1 else 1e-5)

    # level 4 (11 variables): random smooth moments, 128^2, flat, 20 steps
    Q0 = inputs.random_moments_2d(128, 128, 4, seed=1, vel=0.25)
    mesh = oracle.Mesh.rect(128, 128, 0, 1, 0, 1, bc=(1, 1, 1, 1))
    for dt_ in (1, 0):
        Qr = rounded(Q0, dt_)
        got = gpu_run(Z, Z.mesh_2d(128, 128), 4, fr, Qr, 20, dt_)
        e64 = rel_l1(got, oracle_run(oracle, mesh, 4, 2, fr, Qr, 20, None))
        record("2D level 4, 128^2, random moments, 20 steps", dt_, e64, None, e64, 1e-12 if dt_ == 1 else 1e-5)

    # config-3 family: triangles, level 3, circular dam into dry land, Manning 0.03, 50 steps (FP32)
    verts, tris = inputs.jittered_delaunay(61, seed=0)
    Q0 = rounded(inputs.circular_dam_tri(verts, tris, 3), 0)
    frm = (2, 0.0, 0.0, 0.03)
    got = gpu_run(Z, Z.mesh_tri(verts, tris, bc=1), 3, frm, Q0, 50, 0)
    mesh = oracle.Mesh.triangles(verts, tris, bc=1)
    e64 = rel_l1(got, oracle_run(oracle, mesh, 3, 2, frm, Q0, 50, None))
    e32 = rel_l1(got, oracle_run(oracle, mesh, 3, 2, frm, Q0, 50, None, store_f32=True))
    record(f"triangles, level 3, {len(tris)} cells, dam into dry land, 50 steps", 0, e64, e32, e32, 1e-5)

    print("\n| case | path | max rel. L1 vs FP64 oracle | vs FP32-state oracle | bar |")
    print("|---|---|---|---|---|")
    for r in rows:
        print("| " + " | ".join(r) + " |")
    assert not fails, fails

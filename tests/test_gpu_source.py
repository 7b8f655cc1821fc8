"""Fully implicit friction (zoomy_source_mode 1) on the GPU against the oracle in the same mode:
structured 2D FP32 and FP64, 1D FP64, triangles FP32, including a stiff thin layer where the
explicit Newtonian term of the default mode is unstable; mode checks."""
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


def run_both(Z, oracle, desc, omesh, level, dim, Q0, nsteps, dtype, fric, bed=None, dt=0.0, perm=None):
    kind, C_, nu, mn = fric
    Qr = rounded(Q0, dtype)
    ctx = Z.Context(desc, level, Z.friction(kind, C=C_, nu=nu, manning_n=mn), dtype=dtype)
    Z.zoomy_source_mode(ctx.ctx, 1)
    Qlib = Qr if perm is None else np.ascontiguousarray(Qr[:, perm])
    Q = to_device(Qlib, dtype)
    ctx.step(Q, nsteps=nsteps, dt=dt)
    got = Q.double().cpu().numpy()
    ctx.close()
    if perm is not None:
        back = np.empty_like(got)
        back[:, perm] = got
        got = back
    md = oracle.Model(level, dim, g=G, h_dry=1e-6, friction=kind, C=C_, nu=nu, manning_n=mn, implicit_source=True)
    ref, _ = oracle.step(md, omesh, Qr, nsteps, dt=dt, bed=bed, store_f32=(dtype == 0))
    return got, ref


@pytest.mark.parametrize("dtype,level", [(0, 2), (0, 4), (1, 3)])
def test_structured_2d(Z, oracle, dtype, level):
    nx, ny = 53, 41
    Q0 = inputs.random_moments_2d(nx, ny, level, seed=level, vel=0.25)
    _, bed = inputs.gaussian_bump_2d(nx, ny, level, seed=7)
    bedr = rounded(bed, dtype)
    got, ref = run_both(Z, oracle, Z.mesh_2d(nx, ny, bc=(1, 0, 1, 1), bathymetry=bedr),
                        oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 0, 1, 1)), level, 2, Q0, 12, dtype,
                        (1, 0.1, 0.05, 0.0), bed=bedr)
    err = rel_l1(got, ref)
    assert np.all(err <= (1e-12 if dtype == 1 else 1e-5)), err


def test_1d_fp64(Z, oracle):
    level, nx = 3, 400
    Q0 = inputs.dambreak_1d(nx, 0.0, 10.0, level=level, u=0.1, alpha=[0.2, -0.1, 0.05])
    got, ref = run_both(Z, oracle, Z.mesh_1d(nx, 0.0, 10.0), oracle.Mesh.line(nx, 0.0, 10.0), level, 1, Q0, 30, 1,
                        (1, 0.1, 0.01, 0.0))
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-12), err


def test_triangles_manning(Z, oracle):
    level = 2
    verts, tris = inputs.jittered_delaunay(40, seed=3)
    Q0 = inputs.circular_dam_tri(verts, tris, level, radius=0.4, h_in=1.5, h_out=0.5)
    ctx = Z.Context(Z.mesh_tri(verts, tris, bc=1), level, Z.friction(2, manning_n=0.03), dtype=0)
    perm = ctx.permutation()
    ctx.close()
    got, ref = run_both(Z, oracle, Z.mesh_tri(verts, tris, bc=1), oracle.Mesh.triangles(verts, tris, bc=1), level,
                        2, Q0, 15, 0, (2, 0.0, 0.0, 0.03), perm=perm)
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-5), err


def test_stiff_thin_layer(Z, oracle):
    """h = 0.02, nu = 0.5: dt nu / h^2 C_kk / M_k reaches ~100 per step; the implicit mode follows the
    oracle and decays, where the default mode's explicit bulk stress blows up."""
    level, n = 3, 24
    X, Y = inputs.centers_2d(n, n)
    h = 0.02 * (1.0 + 0.1 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y))
    Q0 = np.zeros((inputs.nvars(level, 2), n * n))
    Q0[0] = h.reshape(-1)
    Q0[inputs.idx_alpha(level, 2, 1)] = 0.05 * Q0[0]
    Q0[inputs.idx_beta(level, 2)] = -0.03 * Q0[0]
    dt = 2e-4
    got, ref = run_both(Z, oracle, Z.mesh_2d(n, n), oracle.Mesh.rect(n, n, 0, 1, 0, 1, bc=(1, 1, 1, 1)), level, 2,
                        Q0, 20, 1, (1, 0.1, 0.5, 0.0), dt=dt)
    err = rel_l1(got[1:], ref[1:])
    assert np.all(err <= 1e-10), err
    assert np.abs(got[1:]).sum() < np.abs(Q0[1:]).sum()
    ctx = Z.Context(Z.mesh_2d(n, n), level, Z.friction(1, C=0.1, nu=0.5), dtype=1)
    Q = to_device(Q0, 1)
    with pytest.raises(Z.ZoomyError):  # explicit bulk stress: the state leaves the finite range
        for _ in range(40):
            ctx.step(Q, nsteps=5, dt=dt)
    ctx.close()


def test_mode_checks(Z):
    ctx = Z.Context(Z.mesh_2d(8, 8), 1, Z.friction(1, C=0.1, nu=0.01), dtype=0)
    for bad in (-1, 2):
        with pytest.raises(Z.ZoomyError):
            Z.zoomy_source_mode(ctx.ctx, bad)
    Z.zoomy_source_mode(ctx.ctx, 1)
    with pytest.raises(Z.ZoomyError):  # the learned closure keeps its own friction treatment
        Z.zoomy_closure_set(ctx.ctx, np.zeros(4998), np.ones(6), np.ones(6), 0.1)
    Z.zoomy_source_mode(ctx.ctx, 0)
    Z.zoomy_closure_set(ctx.ctx, np.zeros(4998), np.ones(6), np.ones(6), 0.1)
    with pytest.raises(Z.ZoomyError):
        Z.zoomy_source_mode(ctx.ctx, 1)
    ctx.close()

"""Second order in space (zoomy_space_order 2) on the GPU against the oracle's second-order scheme:
structured 2D FP64 and FP32 with bathymetry and walls, wet/dry fronts with Manning friction, the 1D
dam break in FP64, the implicit friction mode combined with order 2, lake at rest bitwise;
argument checks."""
import numpy as np
import pytest

from gpu_util import rel_l1, rel_max, rounded, to_device
from paper_2601_04826_gb300 import inputs

pytestmark = pytest.mark.gpu
G = 9.81
CFL = 0.3


@pytest.fixture(scope="module")
def Z():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04826_gb300 import build, zoomy

    build.build()
    return zoomy


def run_both(Z, oracle, desc, omesh, level, dim, Q0, nsteps, dtype, fric, bed=None, dt=0.0, implicit=False):
    kind, C_, nu, mn = fric
    Qr = rounded(Q0, dtype)
    ctx = Z.Context(desc, level, Z.friction(kind, C=C_, nu=nu, manning_n=mn), cfl=CFL, dtype=dtype)
    Z.zoomy_space_order(ctx.ctx, 2)
    if implicit:
        Z.zoomy_source_mode(ctx.ctx, 1)
    Q = to_device(Qr, dtype)
    tg = ctx.step(Q, nsteps=nsteps, dt=dt)
    got = Q.double().cpu().numpy()
    ctx.close()
    md = oracle.Model(level, dim, g=G, h_dry=1e-6, friction=kind, C=C_, nu=nu, manning_n=mn, order=2,
                      implicit_source=implicit)
    ref, tr = oracle.step(md, omesh, Qr, nsteps, dt=dt, cfl=CFL, bed=bed, store_f32=(dtype == 0))
    return got, ref, tg, tr


@pytest.mark.parametrize("dtype,level", [(1, 2), (0, 3), (0, 1)])
def test_structured_2d(Z, oracle, dtype, level):
    nx, ny = 57, 43
    Q0 = inputs.random_moments_2d(nx, ny, level, seed=level + 10, vel=0.25)
    _, bed = inputs.gaussian_bump_2d(nx, ny, level, seed=3)
    bedr = rounded(bed, dtype)
    got, ref, tg, tr = run_both(Z, oracle, Z.mesh_2d(nx, ny, bc=(1, 0, 1, 1), bathymetry=bedr),
                                oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 0, 1, 1)), level, 2, Q0, 15, dtype,
                                (1, 0.1, 0.01, 0.0), bed=bedr)
    err = rel_l1(got, ref)
    assert np.all(err <= (1e-12 if dtype == 1 else 1e-5)), err
    assert tg == pytest.approx(tr, rel=1e-12 if dtype == 1 else 1e-5)


@pytest.mark.parametrize("dtype,level,nx,ny,bc", [(0, 0, 1, 37, (0, 1, 1, 0)), (1, 4, 29, 9, (1, 1, 0, 0)),
                                                   (0, 4, 85, 17, (0, 0, 1, 1)), (1, 1, 30, 1, (1, 0, 1, 0)),
                                                   (0, 2, 56, 70, (1, 1, 1, 1)), (1, 3, 3, 2, (0, 1, 0, 1))])
def test_structured_2d_shapes(Z, oracle, dtype, level, nx, ny, bc):
    """Strip and segment edges of the row-marching kernel: one column, one row, widths at, below and above
    multiples of the 28-column strip, every wall / transmissive mix, levels 0 and 4, every output
    element-wise as well."""
    Q0 = inputs.random_moments_2d(nx, ny, level, seed=7 * level + nx, vel=0.25)
    _, bed = inputs.gaussian_bump_2d(nx, ny, level, seed=4)
    bedr = rounded(bed, dtype)
    got, ref, tg, tr = run_both(Z, oracle, Z.mesh_2d(nx, ny, bc=bc, bathymetry=bedr),
                                oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=bc), level, 2, Q0, 12, dtype,
                                (1, 0.1, 0.01, 0.0), bed=bedr)
    tol = 1e-12 if dtype == 1 else 1e-5
    assert np.all(rel_l1(got, ref) <= tol), rel_l1(got, ref)
    assert np.all(rel_max(got, ref) <= (1e-11 if dtype == 1 else 1e-4)), rel_max(got, ref)
    assert tg == pytest.approx(tr, rel=1e-12 if dtype == 1 else 1e-5)


def test_wet_dry_manning_fp32(Z, oracle):
    level, nx, ny = 2, 64, 48
    X, Y = inputs.centers_2d(nx, ny)
    Q0 = np.zeros((inputs.nvars(level, 2), nx * ny))
    Q0[0] = np.where((X - 0.4) ** 2 + (Y - 0.5) ** 2 < 0.04, 1.2, 0.0).reshape(-1)
    got, ref, _, _ = run_both(Z, oracle, Z.mesh_2d(nx, ny), oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 1, 1, 1)),
                              level, 2, Q0, 25, 0, (2, 0.0, 0.0, 0.03))
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-5), err
    assert np.all(got[0] >= 0.0)


def test_dambreak_1d_fp64(Z, oracle):
    level, nx = 1, 2000
    Q0 = inputs.dambreak_1d(nx, 0.0, 10.0, h_left=2.0, h_right=1.0, x_dam=5.0, level=level)
    got, ref, tg, tr = run_both(Z, oracle, Z.mesh_1d(nx, 0.0, 10.0), oracle.Mesh.line(nx, 0.0, 10.0), level, 1, Q0,
                                100, 1, (1, 0.1, 0.01, 0.0))
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-12), err
    assert tg == pytest.approx(tr, rel=1e-12)


def test_order2_with_implicit_friction(Z, oracle):
    level, nx, ny = 3, 40, 36
    Q0 = inputs.random_moments_2d(nx, ny, level, seed=21, vel=0.2)
    got, ref, _, _ = run_both(Z, oracle, Z.mesh_2d(nx, ny), oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 1, 1, 1)),
                              level, 2, Q0, 10, 1, (1, 0.2, 0.05, 0.0), implicit=True)
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("dtype", [0, 1])
def test_lake_at_rest_bitwise(Z, dtype):
    level, nx, ny = 2, 40, 32
    Q0, b = inputs.lake_at_rest_dyadic(nx, ny, level, seed=5)
    ctx = Z.Context(Z.mesh_2d(nx, ny, bathymetry=b), level, Z.friction(1, C=0.1, nu=0.01), cfl=CFL, dtype=dtype)
    Z.zoomy_space_order(ctx.ctx, 2)
    Q = to_device(Q0, dtype)
    ctx.step(Q, nsteps=100, dt=1e-4)
    got = Q.double().cpu().numpy()
    ctx.close()
    np.testing.assert_array_equal(got[0], Q0[0])
    np.testing.assert_array_equal(got[1:], 0.0)


def test_order_checks(Z):
    verts, tris = inputs.jittered_delaunay(8, seed=0)
    ctx = Z.Context(Z.mesh_tri(verts, tris), 1, Z.friction(0), dtype=0)
    with pytest.raises(Z.ZoomyError):
        Z.zoomy_space_order(ctx.ctx, 2)
    ctx.close()
    ctx = Z.Context(Z.mesh_2d(8, 8), 1, Z.friction(1, C=0.1, nu=0.01), dtype=0)
    for bad in (0, 3):
        with pytest.raises(Z.ZoomyError):
            Z.zoomy_space_order(ctx.ctx, bad)
    Z.zoomy_space_order(ctx.ctx, 2)
    with pytest.raises(Z.ZoomyError):
        Z.zoomy_closure_set(ctx.ctx, np.zeros(4998), np.ones(6), np.ones(6), 0.1)
    ctx.close()


def test_full_size_order2(Z, oracle):
    """The timed second-order workload's size and launch configuration: 2048^2 level 2, FP32, the bench's
    bathymetry and surface bump with a background flow and non-zero moments, two steps at CFL 0.45,
    against the oracle's FP32-state form and its FP64 form."""
    n, level = 2048, 2
    Q0, bed = inputs.gaussian_bump_2d(n, n, level, seed=0)
    h = Q0[0]
    for v, a in [(1, 0.3), (2, -0.2), (3, 0.1), (4, -0.05), (5, 0.05), (6, 0.02)]:
        Q0[v] = h * a
    Qr, bedr = rounded(Q0, 0), rounded(bed, 0)
    ctx = Z.Context(Z.mesh_2d(n, n, bathymetry=bedr), level, Z.friction(1, C=0.1, nu=0.01), cfl=0.45, dtype=0)
    Z.zoomy_space_order(ctx.ctx, 2)
    Q = to_device(Qr, 0)
    tg = ctx.step(Q, nsteps=2, dt=0.0)
    got = Q.double().cpu().numpy()
    ctx.close()
    md = oracle.Model(level, 2, g=G, h_dry=1e-6, friction=1, C=0.1, nu=0.01, order=2)
    omesh = oracle.Mesh.rect(n, n, 0, 1, 0, 1, bc=(1, 1, 1, 1))
    ref32, tr = oracle.step(md, omesh, Qr, 2, dt=0.0, cfl=0.45, bed=bedr, store_f32=True)
    ref64, _ = oracle.step(md, omesh, Qr, 2, dt=0.0, cfl=0.45, bed=bedr)
    err32, err64 = rel_l1(got, ref32), rel_l1(got, ref64)
    emax32, emax64 = rel_max(got, ref32), rel_max(got, ref64)
    print("relative L1 vs FP32-storage oracle", err32, "vs FP64 oracle", err64)
    print("element-wise vs FP32-storage oracle", emax32, "vs FP64 oracle", emax64)
    assert tg == pytest.approx(tr, rel=1e-5)
    assert np.all(err32 <= 1e-5), err32
    assert np.all(err64 <= 1e-5), err64
    assert np.all(emax32 <= 1e-5), emax32
    assert np.all(emax64 <= 1e-5), emax64

"""GPU parity of the triangle-mesh path (cell-centric gather kernel, Morton-ordered cells) against
the FP64 CPU oracle, which builds its own neighbours and geometry from the same vertices and
triangles.  The library's cells are in its own order: zoomy_mesh_permutation maps them back."""
import numpy as np
import pytest

from gpu_util import rel_l1, rel_max, rounded, to_device
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


def run_tri(Z, oracle, verts, tris, level, Q0, nsteps, dt=0.0, fric=(2, 0.0, 0.0, 0.03), bed=None, bc=1,
            store_f32=False):
    kind, C_, nu, mn = fric
    ctx = Z.Context(Z.mesh_tri(verts, tris, bc=bc, bathymetry=bed), level, Z.friction(kind, C=C_, nu=nu,
                                                                                      manning_n=mn), dtype=0)
    perm = ctx.permutation()
    assert np.array_equal(np.sort(perm), np.arange(len(tris)))
    Q0r = rounded(Q0, 0)
    Q = to_device(Q0r[:, perm], 0)
    tg = ctx.step(Q, nsteps=nsteps, dt=dt)
    got = np.empty_like(Q0r)
    got[:, perm] = Q.double().cpu().numpy()
    ctx.close()
    md = oracle.Model(level, 2, g=G, h_dry=1e-6, friction=kind, C=C_, nu=nu, manning_n=mn)
    mesh = oracle.Mesh.triangles(verts, tris, bc=bc)
    ref, tr = oracle.step(md, mesh, Q0r, nsteps, dt=dt, cfl=0.45, bed=None if bed is None else rounded(bed, 0),
                          store_f32=store_f32)
    return got, ref, tg, tr


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_tri_dambreak_wet_dry(Z, oracle, level):
    verts, tris = inputs.jittered_delaunay(41, seed=level)
    Q0 = inputs.circular_dam_tri(verts, tris, level, radius=0.4)
    got, ref, tg, tr = run_tri(Z, oracle, verts, tris, level, Q0, 30)
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-5), err
    assert tg == pytest.approx(tr, rel=1e-5)
    assert np.all(got[0] >= 0.0)


@pytest.mark.parametrize("level", [1, 3])
def test_tri_moments_bathymetry_transmissive(Z, oracle, level):
    verts, tris = inputs.jittered_delaunay(37, seed=10 + level)
    c = inputs.tri_centroids(verts, tris)
    rng = np.random.default_rng(level)
    bed = 0.1 * np.sin(2.0 * c[:, 0]) * np.cos(3.0 * c[:, 1])
    h = 1.0 - bed + 0.2 * np.exp(-((c[:, 0] - 0.2) ** 2 + (c[:, 1] + 0.1) ** 2) / 0.05)
    Q0 = np.zeros((inputs.nvars(level, 2), len(tris)))
    Q0[0] = h
    for v in range(1, Q0.shape[0]):
        Q0[v] = h * rng.uniform(-0.2, 0.2) * (1 + 0.3 * np.sin(5 * c[:, 0] + v))
    got, ref, tg, tr = run_tri(Z, oracle, verts, tris, level, Q0, 25, fric=(1, 0.05, 0.01, 0.0), bed=bed, bc=0)
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-5), err


def test_tri_mass_wavespeed_and_locality(Z, oracle):
    level = 3
    verts, tris = inputs.jittered_delaunay(60, seed=4)
    Q0 = rounded(inputs.circular_dam_tri(verts, tris, level, radius=0.3), 0)
    ctx = Z.Context(Z.mesh_tri(verts, tris, bc=1), level, Z.friction(2, manning_n=0.03), dtype=0)
    perm = ctx.permutation()
    Q = to_device(Q0[:, perm], 0)
    md = oracle.Model(level, 2, g=G, h_dry=1e-6, friction=2, manning_n=0.03)
    mesh = oracle.Mesh.triangles(verts, tris, bc=1)
    assert ctx.max_wavespeed(Q) == pytest.approx(oracle.max_wavespeed(md, mesh, Q0), rel=2e-6)
    m0 = ctx.mass(Q)
    assert m0 == pytest.approx(oracle.mass(mesh, Q0), rel=1e-13)
    ctx.step(Q, nsteps=60, dt=0.0)
    assert abs(ctx.mass(Q) - m0) / m0 < 1e-5
    _, dmin = Z.zoomy_mesh_info(ctx.ctx)
    assert dmin == pytest.approx(mesh.min_delta(), rel=1e-12)
    ctx.close()
    # Morton order: centroids of consecutive cells are close
    c = inputs.tri_centroids(verts, tris)[perm]
    step = np.hypot(*np.diff(c, axis=0).T)
    assert np.median(step) < 3.0 * np.sqrt(4.0 / len(tris))


def test_tri_full_size_config3(Z, oracle):
    """~4M-triangle jittered Delaunay mesh, level 3, Manning n = 0.03, circular dam h = 1.5 inside
    r = 0.2 with a dry outside, walls: every output after 2 CFL steps against the oracle."""
    level = 3
    verts, tris = inputs.jittered_delaunay(1415, seed=0)
    assert len(tris) > 3.9e6
    Q0 = inputs.circular_dam_tri(verts, tris, level, radius=0.2, h_in=1.5)
    got, ref32, tg, tr = run_tri(Z, oracle, verts, tris, level, Q0, 2, store_f32=True)
    err, emax = rel_l1(got, ref32), rel_max(got, ref32)
    print("relative L1 vs FP32-storage oracle", err, "element-wise", emax)
    worst = np.argmax(np.abs(got - ref32), axis=1)
    print("worst cells", worst, "h there", ref32[0, worst], "got", got[0, worst])
    assert np.all(err <= 1e-5), err
    assert np.all(emax <= 1e-5), emax

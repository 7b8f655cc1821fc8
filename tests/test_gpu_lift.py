"""The lifting kernel (zoomy_lift3d) against the oracle's lifting: structured 2D (FP32 and FP64, with
bathymetry and dry cells), 1D FP64 and triangles (FP32, library cell order mapped back), all at
several sigma levels including the bed and the surface; argument checks."""
import numpy as np
import pytest

from gpu_util import rounded, to_device
from paper_2601_04826_gb300 import inputs

pytestmark = pytest.mark.gpu
G = 9.81
ZETA = np.array([0.0, 0.1, 0.35, 0.5, 0.8, 1.0])


@pytest.fixture(scope="module")
def Z():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04826_gb300 import build, zoomy

    build.build()
    return zoomy


def lift_gpu(Z, ctx, Q, dtype, zeta=ZETA):
    import torch

    Qd = to_device(Q, dtype)
    K, nc = len(zeta), Q.shape[1]
    out = torch.full((4 * K, nc + 3), float("nan"), dtype=Qd.dtype, device="cuda")  # ldo > nc
    Z.zoomy_lift3d(ctx.ctx, Qd, Qd.stride(0), zeta, out, out.stride(0))
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    assert np.all(np.isnan(got[:, nc:]))  # nothing beyond the cells
    return got[:, :nc].reshape(4, K, nc)


def check(got, ref, tol):
    for f in range(4):
        scale = max(np.abs(ref[f]).max(), 1e-30)
        err = np.abs(got[f] - ref[f]).max() / scale
        assert err <= tol, (f, err)


@pytest.mark.parametrize("dtype", [0, 1])
def test_lift_structured_with_bed_and_dry_cells(Z, oracle, dtype):
    level, nx, ny = 2, 61, 47
    Q = inputs.random_moments_2d(nx, ny, level, seed=4, vel=0.3)
    _, bed = inputs.gaussian_bump_2d(nx, ny, level, seed=9)
    Q[:, [7, 100, 2000]] = 0.0  # dry cells
    Qr, bedr = rounded(Q, dtype), rounded(bed, dtype)
    ctx = Z.Context(Z.mesh_2d(nx, ny, bathymetry=bedr), level, Z.friction(1, C=0.1, nu=0.01), dtype=dtype)
    got = lift_gpu(Z, ctx, Qr, dtype)
    ctx.close()
    ref = oracle.lift3d(oracle.Model(level, 2, g=G), oracle.Mesh.rect(nx, ny, 0, 1, 0, 1), Qr, ZETA, bed=bedr)
    check(got, ref, 1e-12 if dtype == 1 else 2e-5)
    assert np.all(got[:3, :, [7, 100, 2000]] == 0.0)


def test_lift_1d_fp64(Z, oracle):
    level, nx = 3, 300
    Q = inputs.dambreak_1d(nx, 0.0, 10.0, level=level, u=0.2, alpha=[0.1, -0.05, 0.02])
    ctx = Z.Context(Z.mesh_1d(nx, 0.0, 10.0), level, Z.friction(1, C=0.1, nu=0.01), dtype=1)
    got = lift_gpu(Z, ctx, Q, 1)
    ctx.close()
    ref = oracle.lift3d(oracle.Model(level, 1, g=G), oracle.Mesh.line(nx, 0.0, 10.0), Q, ZETA)
    check(got, ref, 1e-12)


def test_lift_triangles(Z, oracle):
    level = 3
    verts, tris = inputs.jittered_delaunay(30, seed=5)
    c = inputs.tri_centroids(verts, tris)
    rng = np.random.default_rng(2)
    Q = np.zeros((inputs.nvars(level, 2), len(tris)))
    Q[0] = 1.0 + 0.3 * np.exp(-((c[:, 0] - 0.1) ** 2 + c[:, 1] ** 2) / 0.1)
    for v in range(1, Q.shape[0]):
        Q[v] = Q[0] * (0.2 * np.sin(3 * c[:, 0] + v) * np.cos(2 * c[:, 1]) + 0.02 * rng.uniform(-1, 1, len(tris)))
    bed = 0.1 * np.cos(2 * c[:, 0]) * np.sin(3 * c[:, 1])
    Qr, bedr = rounded(Q, 0), rounded(bed, 0)
    ctx = Z.Context(Z.mesh_tri(verts, tris, bc=1, bathymetry=bedr), level, Z.friction(1, C=0.1, nu=0.01), dtype=0)
    perm = ctx.permutation()
    got_lib = lift_gpu(Z, ctx, np.ascontiguousarray(Qr[:, perm]), 0)
    ctx.close()
    got = np.empty_like(got_lib)
    got[:, :, perm] = got_lib
    ref = oracle.lift3d(oracle.Model(level, 2, g=G), oracle.Mesh.triangles(verts, tris, bc=1), Qr, ZETA, bed=bedr)
    check(got, ref, 2e-5)


def test_lift_argument_checks(Z):
    import torch

    ctx = Z.Context(Z.mesh_2d(8, 8), 1, Z.friction(0), dtype=0)
    Q = torch.zeros((5, 64), device="cuda")
    Q[0] = 1.0  # lake of depth 1 at rest
    out = torch.zeros((4 * 65, 64), device="cuda")
    for zeta, ldo in (([], 64), (np.linspace(0, 1, 65), 64), ([0.5, 1.2], 64), ([-0.1], 64), ([0.5], 63)):
        with pytest.raises(Z.ZoomyError) as e:
            Z.zoomy_lift3d(ctx.ctx, Q, 64, zeta, out, ldo)
        assert e.value.status == Z.ZOOMY_EINVAL
    Z.zoomy_lift3d(ctx.ctx, Q, 64, [0.0, 1.0], out, 64)
    torch.cuda.synchronize()
    o = out[:8].cpu().numpy().reshape(4, 2, 64)
    assert np.all(o[:3] == 0.0) and np.allclose(o[3, 0], G) and np.all(o[3, 1] == 0.0)
    ctx.close()


def test_lift_full_size(Z, oracle):
    """The timed lifting workload's size and launch configuration: 2048^2 level 2, FP32, 16 sigma levels,
    a moving state over the bench's bathymetry; every output against the oracle."""
    level, n = 2, 2048
    _, bed = inputs.gaussian_bump_2d(n, n, level, seed=0)
    Q = inputs.random_moments_2d(n, n, level, seed=8, vel=0.3)
    Qr, bedr = rounded(Q, 0), rounded(bed, 0)
    zeta = np.linspace(0.0, 1.0, 16)
    ctx = Z.Context(Z.mesh_2d(n, n, bathymetry=bedr), level, Z.friction(1, C=0.1, nu=0.01), dtype=0)
    got = lift_gpu(Z, ctx, Qr, 0, zeta=zeta)
    ctx.close()
    ref = oracle.lift3d(oracle.Model(level, 2, g=G), oracle.Mesh.rect(n, n, 0, 1, 0, 1), Qr, zeta, bed=bedr)
    check(got, ref, 2e-5)

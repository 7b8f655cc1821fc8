"""GPU parity of the fused structured-grid SSP-RK2 step against the FP64 CPU oracle.

All device work goes through the C ABI (libzoomy.so).  Tolerances (relative L1 per
variable after the run): 1e-12 for the FP64 path, 1e-5 for the FP32-state path.
Sizes are chosen to span several warps, strips and row segments with ragged tails.
"""
import numpy as np
import pytest

from gpu_util import rel_l1, rel_max, rounded, to_device
from paper_2601_04826_gb300 import inputs

pytestmark = pytest.mark.gpu

G = 9.81
TOL = {0: 1e-5, 1: 1e-12}


@pytest.fixture(scope="module")
def Z():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04826_gb300 import build, zoomy

    build.build()
    return zoomy


def run_both(Z, oracle, *, dim, level, Q0, bed, dtype, nsteps, dt, fric, mesh_kw, tune=None, cfl=0.45, h_dry=1e-6):
    Q0r = rounded(Q0, dtype)
    bedr = None if bed is None else rounded(bed, dtype)
    if dim == 1:
        desc = Z.mesh_1d(mesh_kw["nx"], mesh_kw["x0"], mesh_kw["x1"], bc=mesh_kw["bc"], bathymetry=bedr)
        omesh = oracle.Mesh.line(mesh_kw["nx"], mesh_kw["x0"], mesh_kw["x1"], *mesh_kw["bc"])
    else:
        desc = Z.mesh_2d(mesh_kw["nx"], mesh_kw["ny"], bc=mesh_kw["bc"], bathymetry=bedr)
        omesh = oracle.Mesh.rect(mesh_kw["nx"], mesh_kw["ny"], 0, 1, 0, 1, bc=mesh_kw["bc"])
    kind, C_, nu, mn = fric
    ctx = Z.Context(desc, level, Z.friction(kind, C=C_, nu=nu, manning_n=mn), g=G, cfl=cfl, h_dry=h_dry,
                    dtype=dtype)
    if tune:
        ctx.tune(*tune)
    Q = to_device(Q0r, dtype)
    t_gpu = ctx.step(Q, nsteps=nsteps, dt=dt)
    got = Q.double().cpu().numpy()
    ctx.close()
    md = oracle.Model(level, dim, g=G, h_dry=h_dry, friction=kind, C=C_, nu=nu, manning_n=mn)
    ref, t_ref = oracle.step(md, omesh, Q0r, nsteps, dt=dt, cfl=cfl, bed=bedr)
    return got, ref, t_gpu, t_ref


def test_config1_dambreak_fp64(Z, oracle):
    """1D level-1 dam break, FP64, 2000 cells on [0,10], slip 0.1 + Newtonian 0.01, 200 CFL steps."""
    Q0 = inputs.dambreak_1d(2000, 0.0, 10.0, 2.0, 1.0, 5.0, level=1)
    got, ref, tg, tr = run_both(Z, oracle, dim=1, level=1, Q0=Q0, bed=None, dtype=1, nsteps=200, dt=0.0,
                                fric=(1, 0.1, 0.01, 0.0), mesh_kw=dict(nx=2000, x0=0.0, x1=10.0, bc=(0, 0)))
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-12), err
    assert tg == pytest.approx(tr, rel=1e-12)


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("dtype", [0, 1])
def test_1d_levels(Z, oracle, level, dtype):
    nx = 777
    Q0 = inputs.dambreak_1d(nx, 0.0, 1.0, 1.6, 0.4, 0.37, level=level, u=0.2,
                            alpha=[0.15 * (-1) ** k / (k + 1) for k in range(level)])
    x = inputs.centers_1d(nx, 0, 1)
    bed = 0.1 * np.sin(2 * np.pi * x)
    got, ref, tg, tr = run_both(Z, oracle, dim=1, level=level, Q0=Q0, bed=bed, dtype=dtype, nsteps=60, dt=0.0,
                                fric=(1, 0.05, 0.01, 0.0), mesh_kw=dict(nx=nx, x0=0.0, x1=1.0, bc=(1, 0)))
    err = rel_l1(got, ref)
    assert np.all(err <= TOL[dtype]), err


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("tune", [(64, 4), (7, 1), (16, 3)])
def test_2d_fp32_levels(Z, oracle, level, tune):
    nx, ny = 97, 61
    Q0 = inputs.random_moments_2d(nx, ny, level, seed=level, vel=0.2)
    _, bed = inputs.gaussian_bump_2d(nx, ny, level, seed=10 + level)
    got, ref, tg, tr = run_both(Z, oracle, dim=2, level=level, Q0=Q0, bed=bed, dtype=0, nsteps=25, dt=0.0,
                                fric=(1, 0.05, 0.01, 0.0), mesh_kw=dict(nx=nx, ny=ny, bc=(1, 0, 0, 1)), tune=tune)
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-5), err
    assert tg == pytest.approx(tr, rel=1e-5)


@pytest.mark.parametrize("level", [1, 2])
def test_2d_fp64(Z, oracle, level):
    nx, ny = 64, 45
    Q0 = inputs.random_moments_2d(nx, ny, level, seed=3, vel=0.25)
    _, bed = inputs.gaussian_bump_2d(nx, ny, level, seed=4)
    got, ref, tg, tr = run_both(Z, oracle, dim=2, level=level, Q0=Q0, bed=bed, dtype=1, nsteps=20, dt=0.0,
                                fric=(1, 0.05, 0.01, 0.0), mesh_kw=dict(nx=nx, ny=ny, bc=(1, 1, 1, 1)),
                                tune=(16, 2))
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-12), err


def test_2d_manning_wet_dry(Z, oracle):
    """Circular dam into dry land with Manning friction: Manning's rank-1 update writes every moment
    row (weights 2k+1), so all seven variables are checked, globally and cell by cell."""
    nx, ny, level = 80, 66, 2
    X, Y = inputs.centers_2d(nx, ny)
    Q0 = np.zeros((inputs.nvars(level, 2), nx * ny))
    Q0[0] = np.where((X - 0.5) ** 2 + (Y - 0.5) ** 2 < 0.04, 1.5, 0.0).reshape(-1)
    got, ref, tg, tr = run_both(Z, oracle, dim=2, level=level, Q0=Q0, bed=None, dtype=0, nsteps=40, dt=0.0,
                                fric=(2, 0.0, 0.0, 0.03), mesh_kw=dict(nx=nx, ny=ny, bc=(1, 1, 1, 1)), tune=(20, 4))
    err, emax = rel_l1(got, ref), rel_max(got, ref)
    assert np.all(err <= 1e-5), err
    assert np.all(emax <= 1e-5), emax
    assert np.all(got[0] >= 0.0)


@pytest.mark.parametrize("dtype", [0, 1])
def test_lake_at_rest_bitwise(Z, oracle, dtype):
    nx, ny, level = 70, 50, 2
    Q0, bed = inputs.lake_at_rest_dyadic(nx, ny, level, seed=5)
    Zc = Z.Context(Z.mesh_2d(nx, ny, bathymetry=bed), level, Z.friction(1, C=0.1, nu=0.01), dtype=dtype)
    Zc.tune(16, 2)
    Q = to_device(Q0, dtype)
    Zc.step(Q, nsteps=500, dt=0.0)
    got = Q.double().cpu().numpy()
    Zc.close()
    np.testing.assert_array_equal(got[0], Q0[0])
    np.testing.assert_array_equal(got[1:], 0.0)


def test_mass_and_wavespeed(Z, oracle):
    nx, ny, level = 90, 77, 3
    Q0 = rounded(inputs.random_moments_2d(nx, ny, level, seed=8), 0)
    _, bed = inputs.gaussian_bump_2d(nx, ny, level, seed=9)
    ctx = Z.Context(Z.mesh_2d(nx, ny, bathymetry=rounded(bed, 0)), level, Z.friction(1, C=0.1, nu=0.01), dtype=0)
    Q = to_device(Q0, 0)
    md = oracle.Model(level, 2, g=G, h_dry=1e-6, friction=1, C=0.1, nu=0.01)
    omesh = oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 1, 1, 1))
    assert ctx.max_wavespeed(Q) == pytest.approx(oracle.max_wavespeed(md, omesh, Q0), rel=2e-6)
    m0 = ctx.mass(Q)
    assert m0 == pytest.approx(oracle.mass(omesh, Q0), rel=1e-14)
    ctx.step(Q, nsteps=100, dt=0.0)
    m1 = ctx.mass(Q)
    assert abs(m1 - m0) / m0 < 1e-5
    ctx.close()


def test_async_steps_accumulate_time_and_match_one_call(Z):
    import torch

    nx, ny, level = 64, 64, 1
    Q0 = inputs.random_moments_2d(nx, ny, level, seed=2)
    a = Z.Context(Z.mesh_2d(nx, ny), level, None, dtype=0)
    Qa = to_device(Q0, 0)
    Qb = Qa.clone()
    for _ in range(5):
        a.step(Qa, nsteps=4, dt=0.0, sync=False)
    t_async = Z.zoomy_sync(a.ctx)
    t_one = a.step(Qb, nsteps=20, dt=0.0)
    assert t_async == pytest.approx(t_one, rel=1e-12)
    assert torch.equal(Qa, Qb)
    a.close()


def test_step_host_matches_device(Z):
    import torch

    nx, ny, level = 50, 40, 2
    Q0 = rounded(inputs.random_moments_2d(nx, ny, level, seed=6), 0)
    ctx = Z.Context(Z.mesh_2d(nx, ny), level, Z.friction(1, C=0.1, nu=0.01), dtype=0)
    Qd = to_device(Q0, 0)
    td = ctx.step(Qd, nsteps=10, dt=0.0)
    Qh = torch.tensor(Q0, dtype=torch.float32).pin_memory()
    th = ctx.step_host(Qh, nsteps=10, dt=0.0)
    assert th == td
    assert torch.equal(Qh, Qd.cpu())
    ctx.close()


def test_deterministic(Z):
    import torch

    nx, ny, level = 128, 96, 2
    Q0 = inputs.random_moments_2d(nx, ny, level, seed=12)
    outs = []
    for _ in range(2):
        ctx = Z.Context(Z.mesh_2d(nx, ny), level, Z.friction(1, C=0.1, nu=0.01), dtype=0)
        Q = to_device(Q0, 0)
        ctx.step(Q, nsteps=30, dt=0.0)
        outs.append(Q.cpu())
        ctx.close()
    assert torch.equal(outs[0], outs[1])


def test_error_paths(Z):
    """Failures are reported as status codes; faults are injected on the host only."""
    import torch

    nx, ny, level = 40, 30, 1
    desc = Z.mesh_2d(nx, ny)
    ctx = Z.zoomy_mesh_create(desc[0])
    Q = torch.zeros((5, nx * ny), device="cuda")
    with pytest.raises(Z.ZoomyError) as e:
        Z.zoomy_step(ctx, Q, nx * ny, 0.0, 1)
    assert e.value.status == Z.ZOOMY_ESTATE
    Z.zoomy_model_set(ctx, level, None, dtype=0)
    with pytest.raises(Z.ZoomyError) as e:
        Z.zoomy_step(ctx, Q, nx * ny - 1, 0.0, 1)
    assert e.value.status == Z.ZOOMY_EINVAL
    # all dry: no wave speed, the CFL step is undefined
    with pytest.raises(Z.ZoomyError) as e:
        Z.zoomy_step(ctx, Q, nx * ny, 0.0, 1)
    assert e.value.status == Z.ZOOMY_ECFL
    # NaN planted in a host-prepared state
    Q0 = inputs.random_moments_2d(nx, ny, level, seed=1)
    Q0[0, 17] = np.nan
    Qn = to_device(Q0, 0)
    with pytest.raises(Z.ZoomyError) as e:
        Z.zoomy_step(ctx, Qn, nx * ny, 1e-4, 3)
    assert e.value.status == Z.ZOOMY_ENAN
    # the status was consumed: a clean state steps again
    Qc = to_device(inputs.random_moments_2d(nx, ny, level, seed=1), 0)
    Z.zoomy_step(ctx, Qc, nx * ny, 0.0, 2)
    Z.zoomy_mesh_destroy(ctx)


def _full_size(Z, oracle, Q0, bed, nsteps, tune):
    n, level = 2048, 2
    Q0r, bedr = rounded(Q0, 0), rounded(bed, 0)
    ctx = Z.Context(Z.mesh_2d(n, n, bathymetry=bedr), level, Z.friction(1, C=0.1, nu=0.01), dtype=0)
    Q = to_device(Q0r, 0)
    if tune:
        ctx.autotune(Q)  # the bench's launch configuration
    ctx.step(Q, nsteps=nsteps, dt=0.0)
    got = Q.double().cpu().numpy()
    ctx.close()
    md = oracle.Model(level, 2, g=G, h_dry=1e-6, friction=1, C=0.1, nu=0.01)
    omesh = oracle.Mesh.rect(n, n, 0, 1, 0, 1, bc=(1, 1, 1, 1))
    ref32, _ = oracle.step(md, omesh, Q0r, nsteps, dt=0.0, cfl=0.45, bed=bedr, store_f32=True)
    ref64, _ = oracle.step(md, omesh, Q0r, nsteps, dt=0.0, cfl=0.45, bed=bedr)
    return got, ref32, ref64


def test_full_size_config2_parity(Z, oracle):
    """2048^2 level-2 FP32 step (autotuned launch configuration, all 29M outputs) on the bench's
    bathymetry and surface bump with a background flow and non-zero moments, against the oracle
    with the state stored in FP32 between stages (FP64 arithmetic) and against the pure FP64 oracle."""
    n, level = 2048, 2
    Q0, bed = inputs.gaussian_bump_2d(n, n, level, seed=0)
    h = Q0[0]
    for v, a in [(1, 0.3), (2, -0.2), (3, 0.1), (4, -0.05), (5, 0.05), (6, 0.02)]:
        Q0[v] = h * a
    got, ref32, ref64 = _full_size(Z, oracle, Q0, bed, 2, tune=True)
    err32, err64 = rel_l1(got, ref32), rel_l1(got, ref64)
    emax32, emax64 = rel_max(got, ref32), rel_max(got, ref64)
    print("relative L1 vs FP32-storage oracle", err32, "vs FP64 oracle", err64)
    print("element-wise vs FP32-storage oracle", emax32, "vs FP64 oracle", emax64)
    assert np.all(err32 <= 1e-5), err32
    assert np.all(err64 <= 1e-5), err64
    # every one of the 29M outputs within 1e-5 of its variable's magnitude
    assert np.all(emax32 <= 1e-5), emax32
    assert np.all(emax64 <= 1e-5), emax64


def test_full_size_bench_state(Z, oracle):
    """The bench's own state (at rest, bump over bathymetry) at 2048^2: depth to 1e-6 relative L1;
    the momenta start at zero, so their error is bounded absolutely against the momentum scale
    h sqrt(g h) ~ 3 (FP32 rounding of the stored depth over the bathymetry makes momentum noise of
    order 1e-8 that no FP32-state scheme reproduces bit for bit)."""
    n, level = 2048, 2
    Q0, bed = inputs.gaussian_bump_2d(n, n, level, seed=0)
    got, ref32, ref64 = _full_size(Z, oracle, Q0, bed, 2, tune=True)
    err = rel_l1(got, ref64)
    print("relative L1 vs FP64 oracle", err, "max abs momentum diff", np.abs(got[1:] - ref64[1:]).max())
    assert err[0] <= 1e-6
    assert rel_max(got[:1], ref64[:1])[0] <= 1e-6
    assert np.abs(got[1:] - ref64[1:]).max() <= 1e-6


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("case", ["slip_bathymetry", "manning_dry"])
def test_decomposition_does_not_change_results(Z, level, case):
    """Every cell is updated by one lane with the same arithmetic whatever the segment height (and
    whether its row is a segment's first, last or an inner row), so the result, the CFL steps
    included, is bitwise independent of the launch configuration: every level, walls on two sides and
    transmissive ones on the others, over bathymetry and across Manning dry fronts."""
    import torch

    nx, ny = 301, 203
    if case == "manning_dry":
        X, Y = inputs.centers_2d(nx, ny)
        Q0 = np.zeros((inputs.nvars(level, 2), nx * ny))
        Q0[0] = np.where((X - 0.4) ** 2 + (Y - 0.55) ** 2 < 0.05, 1.2, 0.0).reshape(-1)
        bed, fr = None, Z.friction(2, manning_n=0.03)
    else:
        Q0 = inputs.random_moments_2d(nx, ny, level, seed=21 + level)
        _, bed = inputs.gaussian_bump_2d(nx, ny, level, seed=22 + level)
        fr = Z.friction(1, C=0.1, nu=0.01)
    outs = []
    for tune in [(8, 1), (64, 1), (203, 1), (17, 4), (5, 1)]:
        ctx = Z.Context(Z.mesh_2d(nx, ny, bc=(1, 0, 0, 1), bathymetry=bed), level, fr, dtype=0)
        ctx.tune(*tune)
        Q = to_device(Q0, 0)
        t = ctx.step(Q, nsteps=5, dt=0.0)
        outs.append((Q.cpu(), t))
        ctx.close()
    for o, t in outs[1:]:
        assert torch.equal(o, outs[0][0]), (o - outs[0][0]).abs().max().item()
        assert t == outs[0][1]


def test_autotune_picks_a_valid_configuration(Z, tmp_path):
    nx, ny, level = 256, 192, 2
    Q0 = inputs.random_moments_2d(nx, ny, level, seed=3)
    ctx = Z.Context(Z.mesh_2d(nx, ny), level, Z.friction(1, C=0.1, nu=0.01), dtype=0)
    Q = to_device(Q0, 0)
    Qc = Q.clone()
    cache = str(tmp_path / "tune.jsonl")
    h, us = ctx.autotune(Q, cache)
    assert 1 <= h <= 256 and us > 0
    import torch

    assert torch.equal(Q, Qc)  # the state is left unchanged
    h2, us2 = ctx.autotune(Q, cache)  # served from the cache
    assert (h2, us2) == (h, pytest.approx(us, rel=1e-3))
    ctx.close()

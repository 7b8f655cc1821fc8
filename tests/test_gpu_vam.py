"""The VAM predictor-corrector on the GPU (zoomy_vam_set) against the oracle: smooth states with walls
and with transmissive ends, flat and over a bed, short and odd lines, the timed workload's size, a
fixed time step, the standing-wave dispersion against linear wave theory, lake at rest (flat and over
a hump, bitwise); mode checks."""
import numpy as np
import pytest

from gpu_util import rel_l1, to_device
from oracle import vam

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


def vam_ctx(Z, n, L, bc, bed=None):
    ctx = Z.Context(Z.mesh_1d(n, 0.0, L, bc=bc, bathymetry=bed), 1, Z.friction(0), g=G, cfl=0.45, dtype=1)
    ctx.vam(True)
    assert ctx.nv == 5
    return ctx


def smooth_state(n, L, seed):
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) * L / n
    Q = np.zeros((5, n))
    Q[0] = 1.0 + 0.15 * np.exp(-((x - 0.45 * L) ** 2) / (0.01 * L * L))
    Q[1] = Q[0] * 0.1 * np.sin(2 * np.pi * x / L)
    Q[2] = Q[0] * 0.03 * np.cos(3 * np.pi * x / L)
    Q[3] = Q[0] * 0.02 * rng.normal(size=n)
    Q[4] = Q[0] * 0.02 * rng.normal(size=n)
    return Q


@pytest.mark.parametrize("bc", [(1, 1), (0, 0), (1, 0)])
def test_matches_oracle(Z, bc):
    n, L, nsteps = 157, 2.0, 25
    Q0 = smooth_state(n, L, seed=sum(bc))
    ctx = vam_ctx(Z, n, L, bc)
    Q = to_device(Q0, 1)
    tg = ctx.step(Q, nsteps=nsteps, dt=0.0)
    got = Q.cpu().numpy()
    ctx.close()
    ref, tr, _ = vam.step(Q0, nsteps, L / n, g=G, bc=bc, cfl=0.45)
    assert tg == pytest.approx(tr, rel=1e-12)
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-10), err


@pytest.mark.parametrize("bc", [(1, 1), (0, 0), (1, 0)])
def test_matches_oracle_over_a_bed(Z, bc):
    """A smooth hump and a ramp under moving water: every b_x term of the predictor and corrector."""
    n, L, nsteps = 157, 2.0, 25
    x = (np.arange(n) + 0.5) * L / n
    bed = 0.25 * np.exp(-((x - 0.7 * L) ** 2) / (0.02 * L * L)) + 0.05 * x / L
    Q0 = smooth_state(n, L, seed=3 + sum(bc))
    Q0[0] = Q0[0] - bed
    for v in range(1, 5):
        Q0[v] = Q0[v] / (Q0[0] + bed) * Q0[0]
    ctx = vam_ctx(Z, n, L, bc, bed)
    Q = to_device(Q0, 1)
    tg = ctx.step(Q, nsteps=nsteps, dt=0.0)
    got = Q.cpu().numpy()
    ctx.close()
    ref, tr, _ = vam.step(Q0, nsteps, L / n, g=G, bc=bc, cfl=0.45, b=bed)
    assert tg == pytest.approx(tr, rel=1e-12)
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-10), err


@pytest.mark.parametrize("bc", [(1, 1), (0, 0)])
def test_lake_at_rest_over_a_hump_bitwise(Z, bc):
    n = 96
    x = (np.arange(n) + 0.5) / n
    bed = np.round(0.25 * np.exp(-((x - 0.4) ** 2) / 0.01) * 2.0**16) / 2.0**16
    Q0 = np.zeros((5, n))
    Q0[0] = 1.0 - bed
    ctx = vam_ctx(Z, n, 1.0, bc, bed)
    Q = to_device(Q0, 1)
    ctx.step(Q, nsteps=40, dt=0.0)
    got = Q.cpu().numpy()
    ctx.close()
    np.testing.assert_array_equal(got, Q0)


@pytest.mark.parametrize("n,bc", [(1, (1, 1)), (2, (0, 1)), (3, (1, 0)), (16, (1, 1)), (33, (0, 0))])
def test_line_lengths(Z, n, bc):
    """Short and odd lines (one block row, a dummy cell, few reduction levels)."""
    L, nsteps = 0.1 * n, 6
    Q0 = smooth_state(n, L, seed=n)
    ctx = vam_ctx(Z, n, L, bc)
    Q = to_device(Q0, 1)
    ctx.step(Q, nsteps=nsteps, dt=0.0)
    got = Q.cpu().numpy()
    ctx.close()
    ref, _, _ = vam.step(Q0, nsteps, L / n, g=G, bc=bc, cfl=0.45)
    # per variable, against its own magnitude (a lone cell between walls keeps momenta at round-off)
    scale = np.maximum(np.abs(ref).max(axis=1), 1e-3)
    err = np.abs(got - ref).max(axis=1) / scale
    assert np.all(err <= 1e-10), err


def test_bench_size(Z):
    """The timed workload's size and launch configuration (2000 cells, 11 reduction levels)."""
    n, L, nsteps = 2000, 20.0, 2
    x = (np.arange(n) + 0.5) * L / n
    Q0 = np.zeros((5, n))
    Q0[0] = 1.0 + 0.2 / np.cosh(np.sqrt(0.75 * 0.2) * (x - 5.0)) ** 2
    Q0[1] = Q0[0] * np.sqrt(G * 1.2) * (1.0 - 1.0 / Q0[0])
    ctx = vam_ctx(Z, n, L, (1, 1))
    Q = to_device(Q0, 1)
    tg = ctx.step(Q, nsteps=nsteps, dt=0.0)
    got = Q.cpu().numpy()
    ctx.close()
    ref, tr, _ = vam.step(Q0, nsteps, L / n, g=G, bc=(1, 1), cfl=0.45)
    assert tg == pytest.approx(tr, rel=1e-12)
    assert np.all(rel_l1(got, ref) <= 1e-10), rel_l1(got, ref)


def test_standing_wave_dispersion(Z):
    H, kH, n = 1.0, 1.0, 200
    k = kH / H
    L = np.pi / k
    x = (np.arange(n) + 0.5) * L / n
    Q0 = np.zeros((5, n))
    Q0[0] = H + 1e-3 * np.cos(k * x)
    ctx = vam_ctx(Z, n, L, (1, 1))
    Q = to_device(Q0, 1)
    hs, ts, t = [Q0[0, 0]], [0.0], 0.0
    for _ in range(2000):
        t += ctx.step(Q, nsteps=1, dt=0.0)
        hs.append(float(Q[0, 0]))
        ts.append(t)
        if hs[-1] < H:
            break
    ctx.close()
    y0, y1 = hs[-2] - H, hs[-1] - H
    tz = ts[-2] + (ts[-1] - ts[-2]) * y0 / (y0 - y1)
    c2 = (np.pi / (2 * tz) / k) ** 2 / (G * H)
    assert abs(c2 - np.tanh(kH) / kH) < 6e-3 * np.tanh(kH) / kH, c2


def test_lake_at_rest_bitwise(Z):
    Q0 = np.zeros((5, 64))
    Q0[0] = 0.7
    ctx = vam_ctx(Z, 64, 1.0, (1, 1))
    Q = to_device(Q0, 1)
    ctx.step(Q, nsteps=30, dt=0.0)
    got = Q.cpu().numpy()
    ctx.close()
    np.testing.assert_array_equal(got, Q0)


def test_fixed_dt(Z):
    """dt > 0: the predictor and the corrector take the given step, not the CFL one."""
    n, L, nsteps, dt = 96, 1.5, 12, 2e-4
    Q0 = smooth_state(n, L, seed=7)
    ctx = vam_ctx(Z, n, L, (1, 0))
    Q = to_device(Q0, 1)
    tg = ctx.step(Q, nsteps=nsteps, dt=dt)
    got = Q.cpu().numpy()
    ctx.close()
    ref, tr, _ = vam.step(Q0, nsteps, L / n, g=G, bc=(1, 0), dt=dt)
    assert tg == pytest.approx(nsteps * dt, rel=1e-12) and tr == pytest.approx(nsteps * dt, rel=1e-12)
    assert np.all(rel_l1(got, ref) <= 1e-10), rel_l1(got, ref)


def test_mode_checks(Z):
    ctx = Z.Context(Z.mesh_2d(8, 8), 1, Z.friction(0), dtype=1)
    with pytest.raises(Z.ZoomyError):
        Z.zoomy_vam_set(ctx.ctx, 1)
    ctx.close()
    ctx = Z.Context(Z.mesh_1d(16, 0.0, 1.0), 1, Z.friction(0), dtype=0)
    with pytest.raises(Z.ZoomyError):  # FP64 only
        Z.zoomy_vam_set(ctx.ctx, 1)
    ctx.close()
    ctx = vam_ctx(Z, 16, 1.0, (1, 1))
    Q = to_device(np.ones((5, 16)), 1)
    with pytest.raises(Z.ZoomyError):
        ctx.max_wavespeed(Q)
    ctx.vam(False)
    assert ctx.nv == 3
    with pytest.raises(Z.ZoomyError):  # enable is 0 or 1
        Z.zoomy_vam_set(ctx.ctx, 2)
    ctx.vam(True)
    Z.zoomy_model_set(ctx.ctx, 2, Z.friction(0), 9.81, 0.45, 1e-6, 1)  # a new model leaves the VAM mode
    assert Z.zoomy_nvars(ctx.ctx) == 4
    ctx.close()


def test_long_line_properties(Z):
    """131072 cells (128-thread CTAs, capped grids, grid-stride loops, 16 reduction levels), beyond the
    oracle's dense solve: properties that hold at any size.  Between walls the mass is conserved, and
    the corrected state satisfies both constraints: R0 and R1 evaluated on it by the oracle's
    residual (central differences, the same ghosts) vanish to round-off relative to their terms."""
    n, L = 131072, 400.0
    dx = L / n
    x = (np.arange(n) + 0.5) * dx
    bed = 0.2 * np.exp(-((x - 0.6 * L) ** 2) / 200.0)
    Q0 = np.zeros((5, n))
    Q0[0] = 1.0 + 0.1 * np.exp(-((x - 0.3 * L) ** 2) / 50.0) - bed
    Q0[1] = 0.1 * Q0[0] * np.sin(2 * np.pi * x / L)
    ctx = vam_ctx(Z, n, L, (1, 1), bed)
    Q = to_device(Q0, 1)
    ctx.step(Q, nsteps=3, dt=0.0)
    got = Q.cpu().numpy()
    ctx.close()
    assert np.all(np.isfinite(got))
    assert abs(got[0].sum() - Q0[0].sum()) / Q0[0].sum() < 1e-13
    bx = vam.bed_slope(bed, dx, (1, 1))[0]
    R = vam.residual(got, np.zeros(2 * n), 0.0, dx, (1, 1), bx)
    h, u0, u1, w0, w1, _ = vam.prim(got)
    scale = np.abs(h * vam.diff(u0, dx, (1, 1), True)).max() + 2.0 * np.abs(w0).max() + 2.0 * np.abs(w1).max()
    assert np.abs(R).max() <= 1e-9 * scale, (np.abs(R).max(), scale)

"""Launch shapes of the first-order 1D line (zoomy_tune_1d): two launches per SSP-RK2 step with 1 to 8
face-centric warps per CTA, or every step of a call in one cooperative launch with grid barriers between
the stages.  The state must be bitwise the same for every shape (one compiled warp body, only the launch
differs), and the persistent launch must match the FP64 oracle like the per-stage launches do.
"""
import numpy as np
import pytest

from gpu_util import rel_l1, rounded, to_device
from paper_2601_04826_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (1, 3), (1, 8), (2, 1), (2, 2), (2, 8)]


@pytest.fixture(scope="module")
def Z():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04826_gb300 import build, zoomy

    build.build()
    return zoomy


def _run(Z, nx, level, dtype, Q0, bed, bc, fric, mode, wpc, calls, nsteps, dt=0.0):
    ctx = Z.Context(Z.mesh_1d(nx, 0.0, 1.0, bc=bc, bathymetry=bed), level, Z.friction(*fric[:1], C=fric[1],
                    nu=fric[2], manning_n=fric[3]), cfl=0.45, h_dry=1e-6, dtype=dtype)
    ctx.tune_1d(mode, wpc)
    Q = to_device(Q0, dtype)
    ts = [ctx.step(Q, nsteps=nsteps, dt=dt) for _ in range(calls)]
    out = Q.cpu()
    ctx.close()
    return out, ts


def _case(nx, level, seed):
    rng = np.random.default_rng(seed)
    Q0 = inputs.dambreak_1d(nx, 0.0, 1.0, 1.6, 0.4, 0.37, level=level, u=0.2,
                            alpha=[0.15 * (-1) ** k / (k + 1) for k in range(level)])
    Q0[0] *= 1.0 + 0.05 * rng.random(nx)
    x = inputs.centers_1d(nx, 0, 1)
    return Q0, 0.1 * np.sin(2 * np.pi * x)


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("nx", [1, 31, 32, 63, 2000, 4099])
def test_shapes_bitwise_equal(Z, level, dtype, nx):
    """Every launch shape gives the same state bits and the same advanced time, for one- and
    many-step calls, ragged CTA tails, a wall and a transmissive end, bathymetry, slip + Newtonian."""
    import torch

    Q0, bed = _case(nx, level, 10 + level)
    Q0r, bedr = rounded(Q0, dtype), rounded(bed, dtype)
    fric = (1, 0.05, 0.01, 0.0)
    ref, tref = _run(Z, nx, level, dtype, Q0r, bedr, (1, 0), fric, 1, 1, 3, 17)
    for mode, wpc in SHAPES[1:] + [(0, 0)]:
        got, t = _run(Z, nx, level, dtype, Q0r, bedr, (1, 0), fric, mode, wpc, 3, 17)
        assert torch.equal(got, ref), (mode, wpc)
        assert t == tref, (mode, wpc)


@pytest.mark.parametrize("fric", [(2, 0.0, 0.0, 0.03), (0, 0.0, 0.0, 0.0)])
def test_shapes_manning_and_frictionless(Z, fric):
    import torch

    nx, level = 1500, 2
    Q0, bed = _case(nx, level, 3)
    Q0[0, :400] = 0.0  # a dry stretch
    for k in range(1, Q0.shape[0]):
        Q0[k, :400] = 0.0
    ref, tref = _run(Z, nx, level, 1, Q0, bed, (0, 1), fric, 1, 1, 2, 25)
    for mode, wpc in [(2, 1), (2, 4), (1, 8)]:
        got, t = _run(Z, nx, level, 1, Q0, bed, (0, 1), fric, mode, wpc, 2, 25)
        assert torch.equal(got, ref), (mode, wpc)
        assert t == tref


@pytest.mark.parametrize("wpc", [1, 4])
def test_persistent_matches_oracle_dambreak(Z, oracle, wpc):
    """The 1D level-1 dam break (2000 cells, FP64, slip 0.1 + Newtonian 0.01) stepped 200 CFL steps in
    one persistent launch against the oracle: relative L1 <= 1e-12 per variable, time to 1e-12."""
    nx = 2000
    Q0 = inputs.dambreak_1d(nx, 0.0, 10.0, 2.0, 1.0, 5.0, level=1)
    ctx = Z.Context(Z.mesh_1d(nx, 0.0, 10.0, bc=(0, 0)), 1, Z.friction(1, C=0.1, nu=0.01), cfl=0.45, dtype=1)
    ctx.tune_1d(Z.LAUNCH_PERSISTENT, wpc)
    Q = to_device(Q0, 1)
    tg = ctx.step(Q, nsteps=200, dt=0.0)
    got = Q.cpu().numpy()
    ctx.close()
    md = oracle.Model(1, 1, g=9.81, h_dry=0.0, friction=1, C=0.1, nu=0.01)
    ref, tr = oracle.step(md, oracle.Mesh.line(nx, 0.0, 10.0, 0, 0), Q0, 200, dt=0.0, cfl=0.45)
    assert np.all(rel_l1(got, ref) <= 1e-12)
    assert tg == pytest.approx(tr, rel=1e-12)


def test_persistent_error_skip_matches_per_stage(Z):
    """A NaN planted in the host-prepared state: both launch shapes report ENAN and leave the same
    bits (the steps after the failing one are skipped in both)."""
    import torch

    nx, level = 900, 1
    Q0, bed = _case(nx, level, 5)
    Q0[0, 450] = np.nan
    outs = []
    for mode, wpc in [(1, 1), (2, 1), (2, 2)]:
        ctx = Z.Context(Z.mesh_1d(nx, 0.0, 1.0, bathymetry=bed), level, Z.friction(1, C=0.05, nu=0.01), dtype=1)
        ctx.tune_1d(mode, wpc)
        Q = to_device(Q0, 1)
        with pytest.raises(Z.ZoomyError) as e:
            ctx.step(Q, nsteps=6, dt=1e-4)
        assert e.value.status == Z.ZOOMY_ENAN
        outs.append(Q.cpu().view(torch.int64))
        ctx.close()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_tune_1d_rejects_bad_values(Z):
    ctx = Z.Context(Z.mesh_1d(100, 0.0, 1.0), 1, None, dtype=1)
    for mode, wpc in [(3, 0), (-1, 0), (0, -1), (0, 9), (1, 32)]:
        with pytest.raises(Z.ZoomyError) as e:
            ctx.tune_1d(mode, wpc)
        assert e.value.status == Z.ZOOMY_EINVAL
    ctx.close()

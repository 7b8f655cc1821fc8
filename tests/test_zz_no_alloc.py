"""The allocation-free step (zoomy_step_noalloc) against the regular entry point.

zoomy_step_noalloc exists for callers that cannot allocate device memory; it keeps its stage
buffer in a fixed array inside the library.  Both entry points launch the same stage kernels, whose
results do not depend on the row decomposition, so the states must agree bitwise and the times
advanced exactly.  This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_util import to_device
from paper_2601_04826_gb300 import inputs

pytestmark = pytest.mark.gpu

NX, NY, LEVEL, BC = 211, 157, 2, (1, 0, 1, 1)


@pytest.fixture(scope="module")
def Z():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04826_gb300 import build, zoomy

    build.build()
    return zoomy


def _case(Z):
    import torch

    Q0 = inputs.random_moments_2d(NX, NY, LEVEL, seed=31, vel=0.2)
    _, bed = inputs.gaussian_bump_2d(NX, NY, LEVEL, seed=32)
    fr = Z.friction(Z.FRICTION_SLIP_NEWTONIAN, C=0.1, nu=0.01)
    ctx = Z.Context(Z.mesh_2d(NX, NY, bc=BC, bathymetry=bed), LEVEL, fr, dtype=Z.FP32)
    bed_dev = torch.tensor(bed, dtype=torch.float32, device="cuda")
    return Q0, fr, ctx, bed_dev


def _noalloc(Z, fr, bed_dev, Q, dt, nsteps, sync=True):
    return Z.zoomy_step_noalloc(NX, NY, 0.0, 1.0, 0.0, 1.0, BC, LEVEL, fr, 9.81, 0.45, 1e-6, bed_dev, Q, NX * NY, dt,
                                nsteps, sync=sync)


@pytest.mark.parametrize("dt", [0.0, 2.5e-4])
def test_noalloc_matches_regular_step_twice(Z, dt):
    import torch

    Q0, fr, ctx, bed_dev = _case(Z)
    Qa = to_device(Q0, 0)
    Qb = Qa.clone()
    for call in range(2):  # two calls in a row: the shared scratch keeps the first call's contents
        ta = ctx.step(Qa, nsteps=6, dt=dt)
        tb = _noalloc(Z, fr, bed_dev, Qb, dt, 6)
        assert torch.equal(Qa, Qb), (call, (Qa - Qb).abs().max().item())
        assert tb == ta, (call, ta, tb)
    ctx.close()


def test_noalloc_clears_status_and_runs_unsynchronised(Z):
    """A call that ends in ENAN leaves the device status flag set in the shared control block; the
    next call must clear it and succeed.  A call without t_advanced (no synchronisation) followed by
    a synchronised one equals two regular calls."""
    import torch

    Q0, fr, ctx, bed_dev = _case(Z)
    bad = to_device(Q0, 0)
    bad[0, NX * (NY // 2) + NX // 2] = float("nan")
    with pytest.raises(Z.ZoomyError) as e:
        _noalloc(Z, fr, bed_dev, bad, 2.5e-4, 2)
    assert e.value.status == Z.ZOOMY_ENAN
    Qa = to_device(Q0, 0)
    Qb = Qa.clone()
    ctx.step(Qa, nsteps=3, dt=0.0)
    ta = ctx.step(Qa, nsteps=4, dt=0.0)
    assert _noalloc(Z, fr, bed_dev, Qb, 0.0, 3, sync=False) is None
    tb = _noalloc(Z, fr, bed_dev, Qb, 0.0, 4)
    assert torch.equal(Qa, Qb), (Qa - Qb).abs().max().item()
    assert tb == ta
    ctx.close()


def test_noalloc_rejects_states_beyond_its_scratch(Z):
    import torch

    nx = ny = 2048  # 7 x 4.2M floats = 117 MB > 32 MiB of scratch
    tiny = torch.zeros(16, device="cuda")
    with pytest.raises(Z.ZoomyError) as e:
        Z.zoomy_step_noalloc(nx, ny, 0.0, 1.0, 0.0, 1.0, (1, 1, 1, 1), 2, None, 9.81, 0.45, 1e-6, tiny, tiny,
                             nx * ny, 0.0, 1)
    assert e.value.status == Z.ZOOMY_EINVAL
    assert "scratch" in str(e.value)


def test_noalloc_rejects_misaligned_state(Z):
    """A state pointer that is not float-aligned is refused before any launch."""
    import torch

    Q0, fr, ctx, bed_dev = _case(Z)
    Q = to_device(Q0, 0)
    before = Q.clone()
    with pytest.raises(Z.ZoomyError) as e:
        _noalloc(Z, fr, bed_dev, Q.data_ptr() + 2, 0.0, 1)
    assert e.value.status == Z.ZOOMY_EINVAL
    assert torch.equal(Q, before)
    ctx.close()

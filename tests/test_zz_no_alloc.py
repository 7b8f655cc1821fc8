"""The allocation-free step (zoomy_step_noalloc) against the regular entry point.

zoomy_step_noalloc exists for callers that cannot allocate device memory; it keeps its stage
buffer in a fixed array inside the library.  This file is collected last so that a run stopping
at its first failure has already run every other test; it also passes on its own in a fresh
process.
"""
import numpy as np
import pytest

from gpu_util import rel_l1, to_device
from paper_2601_04826_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Z():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04826_gb300 import build, zoomy

    build.build()
    return zoomy


def test_noalloc_matches_regular_step_twice(Z):
    import torch

    nx, ny, level, nsteps = 211, 157, 2, 6
    Q0 = inputs.random_moments_2d(nx, ny, level, seed=31, vel=0.2)
    _, bed = inputs.gaussian_bump_2d(nx, ny, level, seed=32)
    bc = (1, 0, 1, 1)
    fr = Z.friction(Z.FRICTION_SLIP_NEWTONIAN, C=0.1, nu=0.01)
    ctx = Z.Context(Z.mesh_2d(nx, ny, bc=bc, bathymetry=bed), level, fr, dtype=Z.FP32)
    Qa = to_device(Q0, 0)
    Qb = Qa.clone()
    bed_dev = torch.tensor(bed, dtype=torch.float32, device="cuda")
    ld = nx * ny
    for call in range(2):  # two calls in a row: the shared scratch keeps the first call's contents
        ta = ctx.step(Qa, nsteps=nsteps, dt=0.0)
        tb = Z.zoomy_step_noalloc(nx, ny, 0.0, 1.0, 0.0, 1.0, bc, level, fr, 9.81, 0.45, 1e-6, bed_dev, Qb, ld,
                                  0.0, nsteps)
        err = rel_l1(Qb.double().cpu().numpy(), Qa.double().cpu().numpy())
        assert np.all(err <= 1e-5), (call, err)
        assert tb == pytest.approx(ta, rel=1e-6)
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

"""Checkpoint / resume: K steps in one zoomy_step call against the same K steps split over two calls,
with the state saved to a host numpy array and reloaded in between (the caller carries t).  With a
fixed dt the split is bitwise invisible on every path.  With the adaptive CFL step the first dt of a
call comes from a wave-speed reduction over the reloaded state, the later ones from the reduction
fused into the previous step; both paths give the same dt, so the split is bitwise invisible too."""
import numpy as np
import pytest

from gpu_util import rounded, to_device
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


def split_vs_whole(Z, make_ctx, Q0, dtype, nsteps, dt, perm=None):
    """(state after nsteps in one call, after nsteps/2 + save/load + nsteps/2, t whole, t split)."""
    Qh = Q0 if perm is None else Q0[:, perm]
    ctx = make_ctx()
    Q = to_device(Qh, dtype)
    t_whole = ctx.step(Q, nsteps=nsteps, dt=dt)
    whole = Q.double().cpu().numpy()
    ctx.close()
    ctx = make_ctx()
    Q = to_device(Qh, dtype)
    t1 = ctx.step(Q, nsteps=nsteps // 2, dt=dt)
    saved = Q.cpu().numpy().copy()  # checkpoint: the state as a host array
    ctx.close()
    ctx = make_ctx()  # a fresh context, as after a restart
    Q = to_device(saved.astype(np.float64), dtype)
    t2 = ctx.step(Q, nsteps=nsteps - nsteps // 2, dt=dt)
    split = Q.double().cpu().numpy()
    ctx.close()
    return whole, split, t_whole, t1 + t2


@pytest.mark.parametrize("dt", [1e-4, 0.0])
def test_resume_structured_fp32(Z, dt):
    Q0, b = inputs.gaussian_bump_2d(96, 80, 2, seed=4)
    Q0, b = rounded(Q0, 0), rounded(b, 0)

    def make():
        return Z.Context(Z.mesh_2d(96, 80, bathymetry=b), 2, Z.friction(1, C=0.1, nu=0.01), dtype=0)

    whole, split, tw, ts = split_vs_whole(Z, make, Q0, 0, 40, dt)
    np.testing.assert_array_equal(split, whole)
    assert ts == pytest.approx(tw, rel=1e-12)


@pytest.mark.parametrize("dt", [1e-4, 0.0])
def test_resume_1d_fp64(Z, dt):
    Q0 = inputs.dambreak_1d(2000, 0.0, 10.0, 2.0, 1.0, 5.0, level=1)

    def make():
        return Z.Context(Z.mesh_1d(2000, 0.0, 10.0), 1, Z.friction(1, C=0.1, nu=0.01), dtype=1)

    whole, split, tw, ts = split_vs_whole(Z, make, Q0, 1, 60, dt)
    np.testing.assert_array_equal(split, whole)
    assert ts == pytest.approx(tw, rel=1e-14)


def test_resume_triangles(Z):
    verts, tris = inputs.jittered_delaunay(41, seed=2)
    Q0 = rounded(inputs.circular_dam_tri(verts, tris, 2), 0)

    def make():
        return Z.Context(Z.mesh_tri(verts, tris, bc=1), 2, Z.friction(2, manning_n=0.03), dtype=0)

    ctx = make()
    perm = ctx.permutation()
    ctx.close()
    whole, split, tw, ts = split_vs_whole(Z, make, Q0, 0, 30, 0.0, perm=perm)
    np.testing.assert_array_equal(split, whole)


def test_resume_vam(Z):
    n, L = 200, 4.0
    x = (np.arange(n) + 0.5) * L / n
    Q0 = np.zeros((5, n))
    Q0[0] = 1.0 + 0.1 * np.exp(-((x - 1.5) ** 2) / 0.1)
    Q0[1] = 0.05 * Q0[0]

    def make():
        ctx = Z.Context(Z.mesh_1d(n, 0.0, L, bc=(1, 0)), 1, Z.friction(0), dtype=1)
        ctx.vam(True)
        return ctx

    whole, split, tw, ts = split_vs_whole(Z, make, Q0, 1, 20, 0.0)
    np.testing.assert_array_equal(split, whole)

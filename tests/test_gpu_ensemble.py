"""Batched ensembles: every member of a ragged ensemble, advanced in one persistent launch (or one
launch per phase, with or without a CUDA graph), equals the same member advanced on its own
through zoomy_step, bit for bit; a small member also matches the FP64 oracle; the bounded grid
barrier reports a timeout instead of hanging."""
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


def single_member(Z, side, C, Qm, level, nsteps, nu=0.01):
    ctx = Z.Context(Z.mesh_2d(side, side), level, Z.friction(1, C=C, nu=nu), dtype=0)
    Q = to_device(Qm, 0)
    t = ctx.step(Q, nsteps=nsteps, dt=0.0)
    out = Q.cpu()
    ctx.close()
    return out, t


SIDES = [33, 64, 47, 90, 31, 128, 61, 5]


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_ensemble_members_equal_single_runs(Z, mode):
    import torch

    level, nsteps = 1, 12
    rng = np.random.default_rng(0)
    slip = rng.lognormal(-2.0, 0.5, len(SIDES))
    Q0, offs = inputs.ensemble_state(SIDES, range(len(SIDES)), level)
    Q0 = rounded(Q0, 0)
    ens = Z.zoomy_ensemble_create(SIDES, slip, level)
    assert np.array_equal(Z.zoomy_ensemble_offsets(ens, len(SIDES)), offs)
    Q = to_device(Q0, 0)
    t = Z.zoomy_ensemble_step(ens, Q, Q.shape[1], nsteps, mode=mode, nmembers=len(SIDES))
    got = Q.cpu()
    Z.zoomy_mesh_destroy(ens)
    for m, s in enumerate(SIDES):
        ref, tm = single_member(Z, s, slip[m], Q0[:, offs[m]:offs[m + 1]], level, nsteps)
        assert torch.equal(got[:, offs[m]:offs[m + 1]], ref), m
        assert t[m] == tm


def test_ensemble_member_matches_oracle(Z, oracle):
    level, nsteps = 1, 15
    sides, slip = [40, 23], [0.2, 0.05]
    Q0, offs = inputs.ensemble_state(sides, [3, 4], level)
    Q0 = rounded(Q0, 0)
    ens = Z.zoomy_ensemble_create(sides, slip, level)
    Q = to_device(Q0, 0)
    Z.zoomy_ensemble_step(ens, Q, Q.shape[1], nsteps, mode=0)
    got = Q.double().cpu().numpy()
    Z.zoomy_mesh_destroy(ens)
    for m, s in enumerate(sides):
        md = oracle.Model(level, 2, g=G, h_dry=1e-6, friction=1, C=slip[m], nu=0.01)
        mesh = oracle.Mesh.rect(s, s, 0, 1, 0, 1, bc=(1, 1, 1, 1))
        ref, _ = oracle.step(md, mesh, Q0[:, offs[m]:offs[m + 1]], nsteps, dt=0.0, cfl=0.45)
        assert np.all(rel_l1(got[:, offs[m]:offs[m + 1]], ref) <= 1e-5)


def test_ensemble_barrier_timeout_is_reported(Z):
    """A barrier waiting for a participant that never arrives gives ETIMEOUT; the context stays usable."""
    level = 1
    Q0, offs = inputs.ensemble_state(SIDES, range(len(SIDES)), level)
    ens = Z.zoomy_ensemble_create(SIDES, [0.1] * len(SIDES), level)
    Q = to_device(Q0, 0)
    Z.zoomy_ensemble_set_barrier(ens, spin_limit=20000, extra_participants=1)
    with pytest.raises(Z.ZoomyError) as e:
        Z.zoomy_ensemble_step(ens, Q, Q.shape[1], 3, mode=1)
    assert e.value.status == Z.ZOOMY_ETIMEOUT
    Z.zoomy_ensemble_set_barrier(ens, spin_limit=20000000, extra_participants=0)
    Q = to_device(Q0, 0)
    Z.zoomy_ensemble_step(ens, Q, Q.shape[1], 3, mode=1)
    Z.zoomy_mesh_destroy(ens)


def test_ensemble_autotune_keeps_state(Z):
    import torch

    level = 1
    Q0, offs = inputs.ensemble_state(SIDES, range(len(SIDES)), level)
    ens = Z.zoomy_ensemble_create(SIDES, [0.1] * len(SIDES), level)
    Q = to_device(Q0, 0)
    Qc = Q.clone()
    h, us = Z.zoomy_ensemble_autotune(ens, Q, Q.shape[1])
    assert h >= 1 and us > 0
    assert torch.equal(Q, Qc)
    Z.zoomy_mesh_destroy(ens)


def test_ensemble_full_size_config4(Z):
    """512 members with sides ~ U{64..512}, slip ~ logNormal(-2, 0.5): 3 persistent steps; sampled
    members (smallest, largest, and five more) equal their single runs bit for bit."""
    import torch

    level, nsteps = 1, 3
    sides, slip, seeds = inputs.ensemble_members(512, seed=0)
    Q0, offs = inputs.ensemble_state(sides, seeds, level)
    Q0 = rounded(Q0, 0)
    ens = Z.zoomy_ensemble_create(sides, slip, level)
    Q = to_device(Q0, 0)
    Z.zoomy_ensemble_autotune(ens, Q, Q.shape[1])
    t = Z.zoomy_ensemble_step(ens, Q, Q.shape[1], nsteps, mode=0, nmembers=512)
    got = Q.cpu()
    Z.zoomy_mesh_destroy(ens)
    pick = sorted({int(np.argmin(sides)), int(np.argmax(sides)), 0, 100, 255, 400, 511})
    for m in pick:
        ref, tm = single_member(Z, int(sides[m]), slip[m], Q0[:, offs[m]:offs[m + 1]], level, nsteps)
        assert torch.equal(got[:, offs[m]:offs[m + 1]], ref), m
        assert t[m] == tm

"""The learned-closure solver on the GPU against the oracle's closure model.

* zero network: the closure kernel reproduces the plain level-1 scheme (oracle and GPU);
* bias-only network (constant predicted moments, exact in BF16): the fused kernel's restricted
  level-4 face terms, Newtonian source and frozen-closure bottom stress match the oracle to 1e-5;
* the tensor-core MLP alone (zoomy_closure_eval) matches the FP64 MLP with BF16 layer inputs within
  a BF16 bound (relative L2 2e-2, cosine >= 0.999);
* a full network: the closed solver matches the oracle within the bound the BF16 MLP allows.
"""
import numpy as np
import pytest

from gpu_util import rel_l1, rel_max, rounded, to_device
from oracle import mlp
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


ENGINES = [0, 1]  # tcgen05 (tensor memory), mma.sync


def run_closure(Z, oracle, params, ins, outs, nx, ny, nsteps, Q0, bed, C=0.1, nu=0.01, bc=(1, 0, 1, 1), engine=0,
                schedule=0):
    Q0r, bedr = rounded(Q0, 0), rounded(bed, 0)
    ctx = Z.Context(Z.mesh_2d(nx, ny, bc=bc, bathymetry=bedr), 1, Z.friction(1, C=C, nu=nu), dtype=0)
    Z.zoomy_closure_set(ctx.ctx, params, ins, outs, C)
    Z.zoomy_closure_engine(ctx.ctx, engine)
    Z.zoomy_closure_schedule(ctx.ctx, schedule)
    Q = to_device(Q0r, 0)
    tg = ctx.step(Q, nsteps=nsteps, dt=0.0)
    got = Q.double().cpu().numpy()
    ctx.close()
    p32 = mlp.unpack(np.asarray(params, dtype=np.float32).astype(np.float64))
    for k in ("W1", "W2", "W3"):  # the kernel holds BF16 weights
        p32[k] = mlp.round_bf16(p32[k])
    cl = oracle.Closure(mlp.pack(p32), np.float32(ins).astype(np.float64), np.float32(outs).astype(np.float64),
                        bf16=True)
    m4 = oracle.Model(4, 2, g=G, h_dry=1e-6, friction=1, C=C, nu=nu)
    mesh = oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=bc)
    ref, tr = oracle.step_closure(m4, cl, mesh, Q0r, nsteps, bed=bedr, schedule=schedule)
    return got, ref, tg, tr


def state(nx, ny, seed):
    Q0 = inputs.random_moments_2d(nx, ny, 1, seed=seed, vel=0.25)
    _, bed = inputs.gaussian_bump_2d(nx, ny, 1, seed=seed + 1)
    return Q0, bed


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("engine", ENGINES)
def test_zero_network_is_level1(Z, oracle, engine, schedule):
    nx, ny = 95, 67
    Q0, bed = state(nx, ny, 1)
    got, ref, tg, tr = run_closure(Z, oracle, np.zeros(mlp.NPARAMS), np.ones(6), np.ones(6), nx, ny, 20, Q0, bed,
                                   engine=engine, schedule=schedule)
    assert np.all(rel_l1(got, ref) <= 1e-5), rel_l1(got, ref)
    m1 = oracle.Model(1, 2, g=G, h_dry=1e-6, friction=1, C=0.1, nu=0.01)
    ref1, _ = oracle.step(m1, oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 0, 1, 1)), rounded(Q0, 0), 20,
                          bed=rounded(bed, 0))
    assert np.all(rel_l1(got, ref1) <= 1e-5)


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("engine", ENGINES)
def test_constant_closure_fv_parity(Z, oracle, engine, schedule):
    nx, ny = 88, 61
    Q0, bed = state(nx, ny, 3)
    p = {k: np.zeros_like(v) for k, v in mlp.init_params(0).items()}
    p["b3"] = np.array([0.125, -0.0625, 0.03125, -0.09375, 0.046875, -0.015625])  # exact in BF16/FP32
    got, ref, tg, tr = run_closure(Z, oracle, mlp.pack(p), np.ones(6), np.ones(6), nx, ny, 20, Q0, bed,
                                   engine=engine, schedule=schedule)
    err, emax = rel_l1(got, ref), rel_max(got, ref)
    assert np.all(err <= 1e-5), err
    assert np.all(emax <= 1e-5), emax
    assert tg == pytest.approx(tr, rel=1e-5)


def test_constant_closure_manning_dry_front(Z, oracle):
    """Manning friction across a dry front with a constant network: the restricted bottom stress with
    the closed moments frozen, the dry cut of the closed profile, walls on every side."""
    nx, ny = 75, 58
    X, Y = inputs.centers_2d(nx, ny)
    Q0 = np.zeros((5, nx * ny))
    Q0[0] = np.where((X - 0.45) ** 2 + (Y - 0.5) ** 2 < 0.06, 1.3, 0.0).reshape(-1)
    Q0[1] = 0.1 * Q0[0]
    Q0[4] = -0.05 * Q0[0]
    p = {k: np.zeros_like(v) for k, v in mlp.init_params(0).items()}
    p["b3"] = np.array([0.0625, -0.03125, 0.015625, -0.046875, 0.0234375, -0.0078125])
    Q0r = rounded(Q0, 0)
    for schedule in (0, 1):
        ctx = Z.Context(Z.mesh_2d(nx, ny, bc=(1, 1, 1, 1)), 1, Z.friction(2, manning_n=0.03), dtype=0)
        Z.zoomy_closure_set(ctx.ctx, mlp.pack(p), np.ones(6), np.ones(6), 0.0)
        Z.zoomy_closure_schedule(ctx.ctx, schedule)
        Q = to_device(Q0r, 0)
        tg = ctx.step(Q, nsteps=30, dt=0.0)
        got = Q.double().cpu().numpy()
        ctx.close()
        cl = oracle.Closure(mlp.pack(p), np.ones(6), np.ones(6), bf16=True)
        m4 = oracle.Model(4, 2, g=G, h_dry=1e-6, friction=2, manning_n=0.03)
        ref, tr = oracle.step_closure(m4, cl, oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 1, 1, 1)), Q0r, 30,
                                      schedule=schedule)
        err, emax = rel_l1(got, ref), rel_max(got, ref)
        assert np.all(err <= 1e-5), (schedule, err)
        assert np.all(emax <= 1e-5), (schedule, emax)
        assert tg == pytest.approx(tr, rel=1e-5)
        assert np.all(got[0] >= 0.0)


@pytest.mark.parametrize("engine", ENGINES)
def test_mlp_eval_matches_oracle(Z, oracle, engine):
    import torch

    rng = np.random.default_rng(2)
    p = mlp.init_params(7)
    for k in p:
        p[k] = p[k] + 0.05 * rng.normal(size=p[k].shape)
    ins = np.array([1.0, 2.0, 2.0, 4.0, 4.0, 5.0])
    outs = np.array([0.1, 0.05, 0.02, 0.1, 0.05, 0.02])
    nx = ny = 16
    ctx = Z.Context(Z.mesh_2d(nx, ny), 1, Z.friction(1, C=0.1, nu=0.01), dtype=0)
    Z.zoomy_closure_set(ctx.ctx, mlp.pack(p), ins, outs, 0.1)
    Z.zoomy_closure_engine(ctx.ctx, engine)
    n = 3001
    F = np.stack([rng.uniform(0.5, 1.5, n), rng.uniform(-0.5, 0.5, n), rng.uniform(-0.5, 0.5, n),
                  rng.uniform(-0.3, 0.3, n), rng.uniform(-0.3, 0.3, n), rng.uniform(0.05, 0.3, n)])
    Fd = torch.tensor(F, dtype=torch.float32, device="cuda")
    Od = torch.zeros_like(Fd)
    Z.zoomy_closure_eval(ctx.ctx, Fd, Od, n)
    Z.zoomy_sync(ctx.ctx)
    got = Od.double().cpu().numpy().T
    ctx.close()
    p32 = mlp.unpack(np.asarray(mlp.pack(p), dtype=np.float32).astype(np.float64))
    for k in ("W1", "W2", "W3"):
        p32[k] = mlp.round_bf16(p32[k])
    ref, _ = mlp.forward(p32, np.float32(F.T).astype(np.float64) * np.float32(ins), bf16_inputs=True)
    ref = ref * np.float32(outs)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    cos = np.sum(got * ref) / (np.linalg.norm(got) * np.linalg.norm(ref))
    assert rel < 2e-2 and cos > 0.999, (rel, cos)


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("engine", ENGINES)
def test_random_network_closed_solver(Z, oracle, engine, schedule):
    nx, ny = 70, 52
    Q0, bed = state(nx, ny, 5)
    rng = np.random.default_rng(11)
    p = mlp.init_params(9)
    for k in p:
        p[k] = 0.5 * p[k] + 0.02 * rng.normal(size=p[k].shape)
    ins = np.array([1.0, 2.0, 2.0, 4.0, 4.0, 5.0])
    outs = np.full(6, 0.05)
    got, ref, tg, tr = run_closure(Z, oracle, mlp.pack(p), ins, outs, nx, ny, 10, Q0, bed, engine=engine,
                                   schedule=schedule)
    err = rel_l1(got, ref)
    print("closed solver relative L1", engine, schedule, err)
    assert np.all(err <= 1e-4), err


def test_engines_agree(Z):
    """tcgen05 and mma.sync evaluate the same BF16 network: they differ only in the FP32 accumulation
    order (and the BF16 rounding of a layer input that lands on the other side of a tie)."""
    import torch

    rng = np.random.default_rng(12)
    p = mlp.init_params(3)
    ins = np.array([1.0, 2.0, 2.0, 4.0, 4.0, 5.0])
    outs = np.full(6, 0.1)
    ctx = Z.Context(Z.mesh_2d(8, 8), 1, Z.friction(1, C=0.1, nu=0.01), dtype=0)
    Z.zoomy_closure_set(ctx.ctx, mlp.pack(p), ins, outs, 0.1)
    n = 128 * 37 + 51  # several tiles per CTA and a ragged last tile
    F = torch.tensor(np.stack([rng.uniform(0.5, 1.5, n), rng.uniform(-0.5, 0.5, n), rng.uniform(-0.5, 0.5, n),
                               rng.uniform(-0.3, 0.3, n), rng.uniform(-0.3, 0.3, n), rng.uniform(0.05, 0.3, n)]),
                     dtype=torch.float32, device="cuda")
    outs_ = []
    for engine in ENGINES:
        Z.zoomy_closure_engine(ctx.ctx, engine)
        O = torch.full_like(F, float("nan"))
        Z.zoomy_closure_eval(ctx.ctx, F, O, n)
        Z.zoomy_sync(ctx.ctx)
        outs_.append(O.double().cpu().numpy())
    ctx.close()
    a, b = outs_
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(b))
    rel = np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel < 2e-3, rel


@pytest.mark.parametrize("schedule", [0, 1])
def test_random_network_full_size(Z, oracle, schedule):
    """The closure workload's size and launch configuration: 1024^2, the tcgen05 engine, a full network,
    two steps, against the oracle's closed level-4 solver with BF16 layer inputs."""
    n = 1024
    Q0, bed = state(n, n, 17)
    rng = np.random.default_rng(19)
    p = mlp.init_params(21)
    for k in p:
        p[k] = 0.5 * p[k] + 0.02 * rng.normal(size=p[k].shape)
    ins = np.array([1.0, 2.0, 2.0, 4.0, 4.0, 5.0])
    outs = np.full(6, 0.05)
    got, ref, tg, tr = run_closure(Z, oracle, mlp.pack(p), ins, outs, n, n, 2, Q0, bed, bc=(1, 1, 1, 1), engine=0,
                                   schedule=schedule)
    err, emax = rel_l1(got, ref), rel_max(got, ref)
    print("closed solver relative L1 at 1024^2", err, "element-wise", emax)
    assert tg == pytest.approx(tr, rel=1e-4)
    assert np.all(err <= 1e-4), err
    # a layer input that sits at a BF16 rounding tie on one side only moves one predicted moment by
    # one BF16 step (2^-8 relative) in that cell: bounded per cell by 1e-3 of each variable's size
    assert np.all(emax <= 1e-3), emax


def test_closed_wavespeed_and_advance(Z, oracle):
    """zoomy_max_wavespeed of a closed context is the level-4 bound on the closed profiles (the speed of
    its CFL step), and zoomy_advance lands on the end time with the CFL steps of that speed."""
    import torch

    nx, ny = 90, 70
    Q0, bed = state(nx, ny, 23)
    rng = np.random.default_rng(29)
    p = mlp.init_params(31)
    for k in p:
        p[k] = 0.5 * p[k] + 0.02 * rng.normal(size=p[k].shape)
    ins, outs = np.array([1.0, 2.0, 2.0, 4.0, 4.0, 5.0]), np.full(6, 0.05)
    Q0r, bedr = rounded(Q0, 0), rounded(bed, 0)
    ctx = Z.Context(Z.mesh_2d(nx, ny, bathymetry=bedr), 1, Z.friction(1, C=0.1, nu=0.01), dtype=0)
    Z.zoomy_closure_set(ctx.ctx, mlp.pack(p), ins, outs, 0.1)
    Q = to_device(Q0r, 0)
    p32 = mlp.unpack(np.asarray(mlp.pack(p), dtype=np.float32).astype(np.float64))
    for k in ("W1", "W2", "W3"):
        p32[k] = mlp.round_bf16(p32[k])
    cl = oracle.Closure(mlp.pack(p32), np.float32(ins).astype(np.float64), np.float32(outs).astype(np.float64),
                        bf16=True)
    m4 = oracle.Model(4, 2, g=G, h_dry=1e-6, friction=1, C=0.1, nu=0.01)
    mesh = oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 1, 1, 1))
    assert ctx.max_wavespeed(Q) == pytest.approx(oracle.closure_max_wavespeed(m4, cl, mesh, Q0r), rel=1e-3)
    T_end = 0.0123
    t, steps = ctx.advance(Q, T_end, chunk=7)
    assert t == pytest.approx(T_end, rel=1e-6)  # the FP32-state path steps with the float of each dt
    dt_cfl = 0.45 * mesh.min_delta() / ctx.max_wavespeed(Q)
    assert steps >= int(T_end / (1.3 * dt_cfl))
    assert torch.isfinite(Q).all()
    ctx.close()

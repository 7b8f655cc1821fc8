"""Pins of the oracle's learned-closure model (CPU):
* the C oracle's closure MLP equals the numpy MLP oracle (itself pinned by finite differences);
* a closure that predicts zero moments reproduces the plain level-1 scheme exactly (the level-4
  terms of the closed moments vanish);
* with constant closed moments, uniform flow follows the closed-form solution of the restricted
  bottom-stress ODE (prognostic moments implicit, closed moments as a frozen forcing)."""
import numpy as np
import pytest
from scipy.linalg import expm

from oracle import mlp
from paper_2601_04826_gb300 import inputs

G = 9.81


def test_c_closure_equals_numpy_mlp(oracle):
    rng = np.random.default_rng(0)
    p = mlp.init_params(5)
    for k in p:
        p[k] = p[k] + 0.1 * rng.normal(size=p[k].shape)
    ins, outs = rng.uniform(0.5, 2.0, 6), rng.uniform(0.1, 1.0, 6)
    X = rng.normal(size=(50, 6))
    for bf16 in (False, True):
        cl = oracle.Closure(mlp.pack(p), ins, outs, bf16=bf16)
        y, _ = mlp.forward(p, X * ins, bf16_inputs=bf16)
        got = np.array([cl.eval(x) for x in X])
        np.testing.assert_allclose(got, y * outs, rtol=1e-12, atol=1e-13)


def zero_closure(oracle):
    return oracle.Closure(np.zeros(mlp.NPARAMS), np.ones(6), np.ones(6), bf16=True)


def test_zero_closure_is_level1(oracle):
    nx, ny = 30, 22
    Q1 = inputs.random_moments_2d(nx, ny, 1, seed=4, vel=0.25)
    _, bed = inputs.gaussian_bump_2d(nx, ny, 1, seed=5)
    mesh = oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 0, 1, 1))
    m1 = oracle.Model(1, 2, g=G, friction=1, C=0.1, nu=0.01)
    m4 = oracle.Model(4, 2, g=G, friction=1, C=0.1, nu=0.01)
    R1, t1 = oracle.step(m1, mesh, Q1, 15, bed=bed)
    Rc, tc = oracle.step_closure(m4, zero_closure(oracle), mesh, Q1, 15, bed=bed)
    np.testing.assert_allclose(Rc, R1, rtol=1e-13, atol=1e-15)
    assert tc == pytest.approx(t1, rel=1e-14)


def test_constant_closure_uniform_flow_ode(oracle):
    """Uniform flow, slip only: d(h alpha_k)/dt = -(2k+1) C/h (h alpha_0 + h alpha_1 + h s_hat), k = 0, 1,
    with s_hat = sum of the three closed moments (constant): y' = -K y - f with the closed form
    y(T) = e^{-KT} y0 - int_0^T e^{-K(T-s)} f ds.  The split scheme converges at first order."""
    h, C, T = 0.7, 0.4, 0.5
    ahat = np.array([0.05, -0.02, 0.01])
    p = {k: np.zeros_like(v) for k, v in mlp.init_params(0).items()}
    p["b3"] = np.concatenate([ahat, [0.0, 0.0, 0.0]])
    cl = oracle.Closure(mlp.pack(p), np.ones(6), np.ones(6), bf16=False)
    m4 = oracle.Model(4, 2, g=G, friction=1, C=C, nu=0.0)
    mesh = oracle.Mesh.rect(3, 3, 0, 1, 0, 1, bc=(0, 0, 0, 0))
    y0 = np.array([0.3, -0.1]) * h
    K = (C / h) * np.array([[1.0, 1.0], [3.0, 3.0]])
    f = (C / h) * h * ahat.sum() * np.array([1.0, 3.0])
    Aug = np.zeros((3, 3))
    Aug[:2, :2] = -K
    Aug[:2, 2] = -f
    yT = (expm(Aug * T) @ np.concatenate([y0, [1.0]]))[:2]
    errs = []
    for n in (40, 80, 160):
        Q = np.zeros((5, 9))
        Q[0] = h
        Q[1] = y0[0]
        Q[3] = y0[1]
        R, _ = oracle.step_closure(m4, cl, mesh, Q, n, dt=T / n)
        assert np.all(R == R[:, :1])
        errs.append(np.max(np.abs(R[[1, 3], 0] - yT)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 0.9), (errs, rates)
    assert errs[-1] < 2e-3 * np.abs(y0).max()


def test_schedule_once_per_step_zero_closure_is_level1(oracle):
    """Schedule 1 (network evaluated once per step on Q^n, held for both stages) with a zero network
    is the plain level-1 scheme exactly, like schedule 0."""
    nx, ny = 30, 22
    Q1 = inputs.random_moments_2d(nx, ny, 1, seed=4, vel=0.25)
    _, bed = inputs.gaussian_bump_2d(nx, ny, 1, seed=5)
    mesh = oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 0, 1, 1))
    m1 = oracle.Model(1, 2, g=G, friction=1, C=0.1, nu=0.01)
    m4 = oracle.Model(4, 2, g=G, friction=1, C=0.1, nu=0.01)
    R1, t1 = oracle.step(m1, mesh, Q1, 15, bed=bed)
    Rc, tc = oracle.step_closure(m4, zero_closure(oracle), mesh, Q1, 15, bed=bed, schedule=1)
    np.testing.assert_allclose(Rc, R1, rtol=1e-13, atol=1e-15)
    assert tc == pytest.approx(t1, rel=1e-14)


@pytest.mark.parametrize("fric", [(1, 0.2, 0.01, 0.0), (2, 0.0, 0.0, 0.03)])
def test_schedule_once_per_step_constant_network_equals_every_stage(oracle, fric):
    """A network whose output does not depend on its input predicts the same moments at Q^n and at
    Q1, so both schedules give bitwise the same states, across a dry front too: a stage input closes
    with its own depth and its own dry cut, whichever state the prediction came from."""
    nx, ny = 28, 24
    X, Y = inputs.centers_2d(nx, ny)
    Q = np.zeros((5, nx * ny))
    Q[0] = np.where((X - 0.45) ** 2 + (Y - 0.5) ** 2 < 0.06, 1.2, 0.0).reshape(-1)
    Q[1] = 0.1 * Q[0]
    Q[3] = -0.05 * Q[0]
    p = {k: np.zeros_like(v) for k, v in mlp.init_params(0).items()}
    p["b3"] = np.array([0.04, -0.02, 0.01, -0.03, 0.015, 0.005])
    cl = oracle.Closure(mlp.pack(p), np.ones(6), np.ones(6), bf16=True)
    kind, C_, nu, mn = fric
    m4 = oracle.Model(4, 2, g=G, friction=kind, C=C_, nu=nu, manning_n=mn)
    mesh = oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 1, 1, 1))
    R0, t0 = oracle.step_closure(m4, cl, mesh, Q, 12, schedule=0)
    R1, t1 = oracle.step_closure(m4, cl, mesh, Q, 12, schedule=1)
    assert np.array_equal(R0, R1)
    assert t0 == t1


def test_schedule_once_per_step_differs_at_first_order(oracle):
    """With a network that depends on the state, holding the step's prediction over stage 2 changes
    the result by O(dt) at a fixed end time (the prediction lags by one stage): the difference
    between the schedules halves with dt, and it is not zero."""
    nx, ny = 20, 16
    Q = inputs.random_moments_2d(nx, ny, 1, seed=9, vel=0.3)
    rng = np.random.default_rng(3)
    p = mlp.init_params(11)
    for k in p:
        p[k] = p[k] + 0.3 * rng.normal(size=p[k].shape)
    cl = oracle.Closure(mlp.pack(p), np.ones(6), np.full(6, 0.2), bf16=False)
    m4 = oracle.Model(4, 2, g=G, friction=1, C=0.1, nu=0.01)
    mesh = oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 1, 1, 1))
    T = 0.02
    diffs = []
    for n in (10, 20, 40):
        R0, _ = oracle.step_closure(m4, cl, mesh, Q, n, dt=T / n, schedule=0)
        R1, _ = oracle.step_closure(m4, cl, mesh, Q, n, dt=T / n, schedule=1)
        diffs.append(np.abs(R1 - R0).max())
    assert diffs[-1] > 0.0
    rates = np.log2(np.array(diffs[:-1]) / np.array(diffs[1:]))
    assert np.all((rates > 0.8) & (rates < 1.3)), (diffs, rates)

"""Pins of the oracle's fully implicit friction (reading R17, the paper's step_source_implicit for
Eq. (PDE-source)): backward Euler on dy/dt = -K y for the moments with the bottom stress and the
Newtonian bulk stress.

* Without viscosity the full solve equals the rank-1 Sherman-Morrison update of the default mode.
* For a spatially uniform state the step is the exact discrete map (I + (I + dt K)^-2) / 2 per
  SSP-RK2 step, with K assembled here from the closed forms M_k = 1/(2k+1), phi_k(0) = 1 and
  C_ik = int phi_i' phi_k' = 2 min(i,k) (min(i,k)+1) for i + k even (0 otherwise).
* In the stiff regime (dt nu / h^2 >> 1) the explicit Newtonian term of the default mode blows up
  while the implicit mode decays monotonically.
"""
import numpy as np
import pytest

from paper_2601_04826_gb300 import inputs

G = 9.81


def K_closed(N, h, C, nu):
    m = N + 1
    K = np.zeros((m, m))
    for k in range(m):
        for i in range(m):
            cik = 2.0 * min(i, k) * (min(i, k) + 1) if (i + k) % 2 == 0 else 0.0
            K[k, i] = (2 * k + 1) * (C / h + nu / h**2 * cik)
    return K


@pytest.mark.parametrize("N", [0, 2, 4])
@pytest.mark.parametrize("fric", [(1, 0.3, 0.0, 0.0), (2, 0.0, 0.0, 0.03)])
def test_without_viscosity_equals_sherman_morrison(oracle, N, fric):
    kind, C, nu, mn = fric
    rng = np.random.default_rng(N)
    me = oracle.Model(N, 2, g=G, friction=kind, C=C, nu=nu, manning_n=mn)
    for _ in range(20):
        y = rng.normal(size=me.nv)
        y[0] = rng.uniform(0.05, 2.0)
        dt = rng.uniform(1e-4, 1.0)
        np.testing.assert_allclose(me.friction_implicit(y, dt), me.bottom_friction(y, dt), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("N", [1, 3])
def test_uniform_flow_is_the_backward_euler_map(oracle, N):
    h, C, nu, dt, nsteps = 0.4, 0.2, 0.05, 0.02, 7
    mesh = oracle.Mesh.rect(3, 3, 0, 1, 0, 1, bc=(0, 0, 0, 0))
    md = oracle.Model(N, 2, g=G, friction=1, C=C, nu=nu, implicit_source=True)
    rng = np.random.default_rng(1)
    a0, b0 = rng.normal(0, 0.3, N + 1), rng.normal(0, 0.3, N + 1)
    Q = np.zeros((inputs.nvars(N, 2), 9))
    Q[0] = h
    for k in range(N + 1):
        Q[inputs.idx_alpha(N, 2, k)] = h * a0[k]
        Q[inputs.idx_beta(N, k)] = h * b0[k]
    R, _ = oracle.step(md, mesh, Q, nsteps, dt=dt)
    A = np.linalg.inv(np.eye(N + 1) + dt * K_closed(N, h, C, nu))
    Mstep = 0.5 * (np.eye(N + 1) + A @ A)
    ya, yb = h * a0, h * b0
    for _ in range(nsteps):
        ya, yb = Mstep @ ya, Mstep @ yb
    got_a = np.array([R[inputs.idx_alpha(N, 2, k), 4] for k in range(N + 1)])
    got_b = np.array([R[inputs.idx_beta(N, k), 4] for k in range(N + 1)])
    np.testing.assert_allclose(got_a, ya, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(got_b, yb, rtol=1e-12, atol=1e-15)
    assert np.all(R[0] == h)


def test_stiff_viscosity_stays_bounded_only_when_implicit(oracle):
    N, h, nu, dt = 3, 0.02, 0.5, 1e-3  # dt nu / h^2 * C_33 (24) * 7 = 210
    mesh = oracle.Mesh.rect(2, 2, 0, 1, 0, 1, bc=(0, 0, 0, 0))
    Q = np.zeros((inputs.nvars(N, 2), 4))
    Q[0] = h
    Q[inputs.idx_alpha(N, 2, 1)] = 0.1 * h
    Q[inputs.idx_alpha(N, 2, 3)] = -0.05 * h
    norms = {}
    for implicit in (False, True):
        md = oracle.Model(N, 2, g=G, friction=1, C=0.0, nu=nu, implicit_source=implicit)
        R = Q.copy()
        hist = [np.abs(R[1:, 0]).sum()]
        for _ in range(10):
            R, _ = oracle.step(md, mesh, R, 1, dt=dt)
            hist.append(np.abs(R[1:, 0]).sum())
        norms[implicit] = np.array(hist)
    assert norms[False][-1] > 1e3 * norms[False][0] or not np.isfinite(norms[False][-1])
    assert np.all(np.diff(norms[True]) <= 1e-15) and norms[True][-1] < norms[True][0]

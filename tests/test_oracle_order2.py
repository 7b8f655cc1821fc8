"""Pins of the oracle's second-order scheme (reading R18: MUSCL with minmod-limited slopes of
(h, eta, velocity moments), hydrostatic reconstruction between reconstructed face states and the
cell-interior pressure and nonconservative terms):

* lake at rest with a dry island stays at rest bitwise (dyadic data), levels 0 and 2;
* mass is conserved in a closed domain;
* a smooth wave converges at second order (first order at first order) against a fine-grid run;
* the Stoker dam break converges, with a smaller error than first order at the same resolution;
* zero moments reduce level N to level 0 bitwise; 2D y-uniform data reproduce 1D; x <-> y symmetry.
"""
import numpy as np
import pytest

from paper_2601_04826_gb300 import inputs

G = 9.81


def run_to(oracle, md, mesh, Q, T, cfl=0.3, bed=None):
    t, n = 0.0, 0
    while t < T - 1e-14:
        dt = min(oracle.cfl_dt(md, mesh, Q, cfl), T - t)
        assert np.isfinite(dt) and dt > 0.0 and n < 50000
        Q, _ = oracle.step(md, mesh, Q, 1, dt=dt, bed=bed)
        t += dt
        n += 1
    return Q


@pytest.mark.parametrize("level", [0, 2])
def test_lake_at_rest_bitwise(oracle, level):
    nx, ny = 24, 20
    Q, b = inputs.lake_at_rest_dyadic(nx, ny, level, seed=5)
    md = oracle.Model(level, 2, g=G, friction=1, C=0.1, nu=0.01, order=2)
    mesh = oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 1, 1, 1))
    R, _ = oracle.step(md, mesh, Q, 200, dt=2e-4, bed=b)
    np.testing.assert_array_equal(R[0], Q[0])
    np.testing.assert_array_equal(R[1:], 0.0)


def test_mass_conserved(oracle):
    nx, ny, level = 28, 24, 2
    Q = inputs.random_moments_2d(nx, ny, level, seed=1)
    _, b = inputs.gaussian_bump_2d(nx, ny, level, seed=2)
    md = oracle.Model(level, 2, g=G, friction=1, C=0.05, nu=0.01, order=2)
    mesh = oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 1, 1, 1))
    m0 = oracle.mass(mesh, Q)
    R, _ = oracle.step(md, mesh, Q, 40, dt=0.0, cfl=0.3, bed=b)
    assert abs(oracle.mass(mesh, R) - m0) / m0 < 1e-13


def _smooth(nx):
    x = inputs.centers_1d(nx, 0.0, 1.0)
    Q = np.zeros((2, nx))
    Q[0] = 1.0 + 0.2 * np.exp(-((x - 0.5) ** 2) / 0.01)
    return Q


def _cell_average(fine, factor):
    return fine.reshape(fine.shape[0], -1, factor).mean(axis=2)


def test_smooth_wave_converges_at_second_order(oracle):
    T, nf = 0.04, 6400
    ref = run_to(oracle, oracle.Model(0, 1, g=G, order=2), oracle.Mesh.line(nf, 0.0, 1.0), _smooth(nf), T)
    errs = {1: [], 2: []}
    sizes = [100, 200, 400, 800]
    for order in (1, 2):
        md = oracle.Model(0, 1, g=G, order=order)
        for nx in sizes:
            R = run_to(oracle, md, oracle.Mesh.line(nx, 0.0, 1.0), _smooth(nx), T)
            avg = _cell_average(ref, nf // nx)
            errs[order].append(np.abs(R[0] - avg[0]).mean())
    r1 = np.log2(np.array(errs[1][:-1]) / np.array(errs[1][1:]))
    r2 = np.log2(np.array(errs[2][:-1]) / np.array(errs[2][1:]))
    assert np.all(r1 < 1.3) and np.all(r1 > 0.7), (errs[1], r1)
    assert np.all(r2 > 1.6), (errs[2], r2)
    assert np.all(np.array(errs[2]) < np.array(errs[1]))


def test_smooth_moment_wave_converges_at_second_order(oracle):
    """Level 2 with moments: the nonconservative product (faces and cell interiors) is exercised."""
    level, T, nf = 2, 0.03, 3200

    def init(nx):
        x = inputs.centers_1d(nx, 0.0, 1.0)
        Q = np.zeros((inputs.nvars(level, 1), nx))
        Q[0] = 1.0 + 0.2 * np.exp(-((x - 0.5) ** 2) / 0.01)
        Q[1] = Q[0] * 0.1 * np.exp(-((x - 0.45) ** 2) / 0.02)
        Q[2] = Q[0] * 0.15 * np.exp(-((x - 0.55) ** 2) / 0.015)
        Q[3] = Q[0] * -0.1 * np.exp(-((x - 0.5) ** 2) / 0.02)
        return Q

    md = oracle.Model(level, 1, g=G, order=2)
    ref = run_to(oracle, md, oracle.Mesh.line(nf, 0.0, 1.0), init(nf), T)
    errs = []
    for nx in (100, 200, 400):
        R = run_to(oracle, md, oracle.Mesh.line(nx, 0.0, 1.0), init(nx), T)
        avg = _cell_average(ref, nf // nx)
        errs.append(np.abs(R - avg).mean(axis=1).sum())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.6), (errs, rates)


def test_stoker_converges(oracle):
    from scipy.optimize import brentq

    T, hl, hr = 0.5, 2.0, 1.0
    cl = np.sqrt(G * hl)
    hm = brentq(lambda h: 2 * (cl - np.sqrt(G * h)) - (h - hr) * np.sqrt(G * (h + hr) / (2 * h * hr)), hr, hl)
    um = 2 * (cl - np.sqrt(G * hm))
    S = hm * um / (hm - hr)

    def exact(x):
        xi = (x - 5.0) / T
        h = np.where(xi <= -cl, hl, (2 * cl - xi) ** 2 / (9 * G))
        h = np.where(xi >= um - np.sqrt(G * hm), hm, h)
        return np.where(xi >= S, hr, h)

    errs = {1: [], 2: []}
    for order in (1, 2):
        md = oracle.Model(0, 1, g=G, h_dry=1e-10, order=order)
        for nx in (250, 500, 1000):
            Q = inputs.dambreak_1d(nx, 0.0, 10.0, h_left=hl, h_right=hr, x_dam=5.0, level=0)
            R = run_to(oracle, md, oracle.Mesh.line(nx, 0.0, 10.0), Q, T)
            errs[order].append(np.abs(R[0] - exact(inputs.centers_1d(nx, 0.0, 10.0))).sum() * 10.0 / nx)
        if order == 2:  # limited slopes: no new extrema across the monotone Riemann fan
            assert R[0].max() <= hl + 1e-12 and R[0].min() >= hr - 1e-12
    rates = np.log2(np.array(errs[2][:-1]) / np.array(errs[2][1:]))
    assert np.all(rates >= 0.5), (errs[2], rates)
    assert np.all(np.array(errs[2]) < np.array(errs[1])), errs


def test_zero_moments_reduce_to_level0(oracle):
    nx = ny = 20
    Q0, b = inputs.gaussian_bump_2d(nx, ny, 0, seed=3)
    Q2 = np.zeros((inputs.nvars(2, 2), nx * ny))
    Q2[:3] = Q0
    mesh = oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(1, 1, 1, 1))
    m0, m2 = oracle.Model(0, 2, g=G, order=2), oracle.Model(2, 2, g=G, order=2)
    dt = 0.2 * mesh.min_delta() / oracle.max_wavespeed(m0, mesh, Q0)
    R0, _ = oracle.step(m0, mesh, Q0, 15, dt=dt, bed=b)
    R2, _ = oracle.step(m2, mesh, Q2, 15, dt=dt, bed=b)
    np.testing.assert_array_equal(R2[:3], R0)
    np.testing.assert_array_equal(R2[3:], 0.0)


def test_y_uniform_2d_is_1d(oracle):
    level, nx, ny = 2, 60, 4
    Q1 = inputs.dambreak_1d(nx, 0.0, 1.0, h_left=1.5, h_right=1.0, x_dam=0.5, level=level, u=0.1,
                            alpha=[0.05, -0.02])
    Q2 = np.zeros((inputs.nvars(level, 2), nx * ny))
    for v1, v2 in zip([0] + [inputs.idx_alpha(level, 1, k) for k in range(level + 1)],
                      [0] + [inputs.idx_alpha(level, 2, k) for k in range(level + 1)]):
        Q2[v2] = np.tile(Q1[v1], ny)
    m1 = oracle.Model(level, 1, g=G, friction=1, C=0.1, nu=0.01, order=2)
    m2 = oracle.Model(level, 2, g=G, friction=1, C=0.1, nu=0.01, order=2)
    R1, _ = oracle.step(m1, oracle.Mesh.line(nx, 0.0, 1.0), Q1, 20, dt=5e-4)
    R2, _ = oracle.step(m2, oracle.Mesh.rect(nx, ny, 0, 1, 0, 1, bc=(0, 0, 1, 1)), Q2, 20, dt=5e-4)
    for v1, v2 in zip([0] + [inputs.idx_alpha(level, 1, k) for k in range(level + 1)],
                      [0] + [inputs.idx_alpha(level, 2, k) for k in range(level + 1)]):
        for j in range(ny):
            np.testing.assert_allclose(R2[v2, j * nx:(j + 1) * nx], R1[v1], rtol=1e-13, atol=1e-14)


def test_transpose_symmetry(oracle):
    level, n = 2, 18
    Q = inputs.random_moments_2d(n, n, level, seed=6)
    _, b = inputs.gaussian_bump_2d(n, n, level, seed=4)
    md = oracle.Model(level, 2, g=G, friction=1, C=0.1, nu=0.01, order=2)
    mesh = oracle.Mesh.rect(n, n, 0, 1, 0, 1, bc=(1, 1, 1, 1))

    def T_(Qx):
        Qt = Qx.reshape(Qx.shape[0], n, n).transpose(0, 2, 1).reshape(Qx.shape[0], -1).copy()
        for k in range(level + 1):
            a, c = inputs.idx_alpha(level, 2, k), inputs.idx_beta(level, k)
            Qt[[a, c]] = Qt[[c, a]]
        return Qt

    bt = b.reshape(n, n).T.reshape(-1).copy()
    R, _ = oracle.step(md, mesh, Q, 10, dt=1e-3, bed=b)
    Rt, _ = oracle.step(md, mesh, T_(Q), 10, dt=1e-3, bed=bt)
    np.testing.assert_allclose(T_(R), Rt, rtol=1e-12, atol=1e-14)

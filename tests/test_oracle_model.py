"""Pins P2-P5 and P11 on the oracle's model functions (flux, NC matrix, wave speed).

* P2  level 0 is the shallow-water system of Sec. 3.1: its flux and its
      eigenvalues u.n, u.n +- sqrt(g h) (the paper's symbolic eigenvalues with
      n.n = 1 and h^5 simplified).
* P3  level 1: the quasilinear matrix dF/dQ + B has the eigenvalues
      u_m, u_m +- sqrt(g h + alpha_1^2) (the known SME-1 spectrum, and the reason
      the k = 0 row of the NC matrix is left out -- with it, level 0 would not be
      the SWE); in 2D the transported beta-moments add u_m +- alpha_1/sqrt(3).
* P4  level 2 at alpha_2 = 0: u_m +- sqrt(g h + alpha_1^2), u_m +- alpha_1/sqrt(5);
      this separates the index order B_kjl of Eq. (sme) from the swapped order of
      the listing in Sec. 2.1.1 (which gives alpha_1/sqrt(3)).
* P5  the wave-speed bound s dominates |Re lambda| on sampled states with real spectra.
* P11 rotation invariance of the 2D flux and spectrum.

dF/dQ is taken by central differences of the oracle's own flux, so these tests
check the flux and NC routines against closed forms, not against themselves.
"""
import numpy as np
import pytest

G = 9.81


def jac(model, q, nx, ny, eps=1e-6):
    nv = len(q)
    J = np.zeros((nv, nv))
    for c in range(nv):
        d = eps * max(1.0, abs(q[c]))
        qp = q.copy()
        qm = q.copy()
        qp[c] += d
        qm[c] -= d
        J[:, c] = (model.flux(qp, nx, ny) - model.flux(qm, nx, ny)) / (2 * d)
    return J


def quasilinear(model, q, nx=1.0, ny=0.0):
    return jac(model, q, nx, ny) + model.nc_matrix(q, nx, ny)


def state_1d(model, h, u, alphas):
    q = np.zeros(model.nv)
    q[0] = h
    q[1] = h * u
    for k, a in enumerate(alphas, start=1):
        q[model.index_alpha(k)] = h * a
    return q


def state_2d(model, h, u, v, alphas, betas):
    q = np.zeros(model.nv)
    q[0] = h
    q[model.index_alpha(0)] = h * u
    q[model.index_beta(0)] = h * v
    for k, a in enumerate(alphas, start=1):
        q[model.index_alpha(k)] = h * a
    for k, b in enumerate(betas, start=1):
        q[model.index_beta(k)] = h * b
    return q


def test_level0_flux_is_swe(oracle):
    md = oracle.Model(0, 2, g=G)
    h, u, v = 1.3, 0.7, -0.4
    q = np.array([h, h * u, h * v])
    Fx = md.flux(q, 1.0, 0.0)
    Fy = md.flux(q, 0.0, 1.0)
    np.testing.assert_allclose(Fx, [h * u, h * u * u + 0.5 * G * h * h, h * u * v], rtol=1e-14)
    np.testing.assert_allclose(Fy, [h * v, h * u * v, h * v * v + 0.5 * G * h * h], rtol=1e-14)
    nx, ny = 0.6, 0.8
    np.testing.assert_allclose(md.flux(q, nx, ny), nx * Fx + ny * Fy, rtol=1e-14)
    np.testing.assert_array_equal(md.nc_matrix(q, nx, ny), np.zeros((3, 3)))


def test_level0_eigenvalues(oracle):
    md = oracle.Model(0, 2, g=G)
    h, u, v = 0.9, 0.4, -1.1
    q = np.array([h, h * u, h * v])
    for th in np.linspace(0, 2 * np.pi, 7):
        n = np.array([np.cos(th), np.sin(th)])
        un = u * n[0] + v * n[1]
        lam = np.sort(np.linalg.eigvals(quasilinear(md, q, *n)).real)
        np.testing.assert_allclose(lam, np.sort([un - np.sqrt(G * h), un, un + np.sqrt(G * h)]), atol=1e-8)
        assert md.wavespeed(q) == pytest.approx(np.hypot(u, v) + np.sqrt(G * h), rel=1e-15)


@pytest.mark.parametrize("h,u,a1", [(1.0, 0.5, 0.3), (2.0, -0.2, 0.8), (0.3, 1.5, -0.4)])
def test_level1_eigenvalues_1d(oracle, h, u, a1):
    md = oracle.Model(1, 1, g=G)
    q = state_1d(md, h, u, [a1])
    lam = np.sort(np.linalg.eigvals(quasilinear(md, q)).real)
    c = np.sqrt(G * h + a1 * a1)
    np.testing.assert_allclose(lam, [u - c, u, u + c], atol=1e-7)
    # the wave-speed bound is the spectral radius at level 1
    assert md.wavespeed(q) == pytest.approx(np.max(np.abs(lam)), rel=1e-7)


def test_level1_eigenvalues_2d(oracle):
    md = oracle.Model(1, 2, g=G)
    h, u, v, a1, b1 = 1.1, 0.5, 0.2, 0.3, -0.25
    q = state_2d(md, h, u, v, [a1], [b1])
    lam = np.sort(np.linalg.eigvals(quasilinear(md, q, 1.0, 0.0)).real)
    c = np.sqrt(G * h + a1 * a1)
    want = np.sort([u - c, u, u + c, u - a1 / np.sqrt(3), u + a1 / np.sqrt(3)])
    np.testing.assert_allclose(lam, want, atol=1e-7)


def test_level1_without_k0_nc_row(oracle):
    """The NC matrix has no k = 0 row and no k = 0 column (reading of Eq. (sme))."""
    for dim in (1, 2):
        md = oracle.Model(3, dim, g=G)
        rng = np.random.default_rng(1)
        q = np.concatenate([[1.2], rng.uniform(-0.5, 0.5, md.nv - 1)])
        Bn = md.nc_matrix(q, 0.6, 0.8 if dim == 2 else 0.0)
        rows0 = [0, md.index_alpha(0)] + ([md.index_beta(0)] if dim == 2 else [])
        assert np.all(Bn[rows0, :] == 0) and np.all(Bn[:, rows0] == 0)


@pytest.mark.parametrize("h,u,a1", [(1.0, 0.5, 0.3), (1.7, -0.4, 0.9)])
def test_level2_eigenvalues_alpha2_zero(oracle, h, u, a1):
    md = oracle.Model(2, 1, g=G)
    q = state_1d(md, h, u, [a1, 0.0])
    lam = np.sort(np.linalg.eigvals(quasilinear(md, q)).real)
    c = np.sqrt(G * h + a1 * a1)
    want = np.sort([u - c, u + c, u - a1 / np.sqrt(5), u + a1 / np.sqrt(5)])
    np.testing.assert_allclose(lam, want, atol=1e-7)


@pytest.mark.parametrize("dim,N", [(1, 2), (1, 3), (1, 4), (2, 2), (2, 3), (2, 4)])
def test_wavespeed_bounds_spectrum(oracle, dim, N):
    md = oracle.Model(N, dim, g=G)
    rng = np.random.default_rng(100 * dim + N)
    n_real = 0
    for _ in range(300):
        h = rng.uniform(0.05, 2.0)
        scale = rng.uniform(0.0, 1.5)
        if dim == 1:
            q = state_1d(md, h, rng.uniform(-1, 1), rng.uniform(-scale, scale, N))
            nrm = (1.0, 0.0)
        else:
            q = state_2d(md, h, rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(-scale, scale, N),
                         rng.uniform(-scale, scale, N))
            th = rng.uniform(0, 2 * np.pi)
            nrm = (np.cos(th), np.sin(th))
        lam = np.linalg.eigvals(quasilinear(md, q, *nrm))
        s = md.wavespeed(q)
        if np.max(np.abs(lam.imag)) < 1e-6 * s:
            n_real += 1
            assert np.max(np.abs(lam.real)) <= s * (1 + 1e-6)
    assert n_real > 50


def rotate_state(md, q, c, s):
    """Velocity moments (a_k, b_k) -> rotated by the angle with cos c, sin s."""
    r = q.copy()
    for k in range(md.N + 1):
        a, b = q[md.index_alpha(k)], q[md.index_beta(k)]
        r[md.index_alpha(k)] = c * a + s * b
        r[md.index_beta(k)] = -s * a + c * b
    return r


@pytest.mark.parametrize("N", [0, 1, 2, 3])
def test_rotation_invariance(oracle, N):
    md = oracle.Model(N, 2, g=G)
    rng = np.random.default_rng(7 + N)
    q = state_2d(md, 1.3, 0.4, -0.3, rng.uniform(-0.3, 0.3, N), rng.uniform(-0.3, 0.3, N))
    th = 0.7
    c, s = np.cos(th), np.sin(th)
    # F_n(Q) = R^-1 F_x(R Q): rotating the frame so that n becomes x
    Fn = md.flux(q, c, s)
    Fx_rot = md.flux(rotate_state(md, q, c, s), 1.0, 0.0)
    np.testing.assert_allclose(rotate_state(md, Fn, c, s), Fx_rot, rtol=1e-12, atol=1e-13)
    la = np.sort_complex(np.linalg.eigvals(quasilinear(md, q, c, s)))
    lb = np.sort_complex(np.linalg.eigvals(quasilinear(md, rotate_state(md, q, c, s), 1.0, 0.0)))
    np.testing.assert_allclose(la, lb, atol=1e-6)
    assert md.wavespeed(q) == pytest.approx(md.wavespeed(rotate_state(md, q, c, s)), rel=1e-14)


def test_dry_state_has_no_velocity(oracle):
    md = oracle.Model(2, 2, g=G, h_dry=1e-6)
    q = np.array([5e-7, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    F = md.flux(q, 1.0, 0.0)
    assert F[0] == 0.0 and F[1] == pytest.approx(0.5 * G * 5e-7**2)
    assert np.all(md.nc_matrix(q, 1.0, 0.0) == 0)
    assert md.wavespeed(q) == pytest.approx(np.sqrt(G * 5e-7))

"""Pins of the oracle's lifting to three-dimensional fields (Sec. "Postprocessing", interpolate_3d):

* the velocity profile is the moment expansion (checked against numpy's Legendre series) and its depth
  average is the mean velocity (Gauss quadrature in zeta);
* at the bed the vertical velocity satisfies no penetration, w = u . grad b (linear bed: exact);
* level 0 on a flat bed reproduces the paper's SWE lifting w = -h (d_x u + d_y v) at the surface
  (linear fields: central differences are exact);
* for smooth fields the vertical velocity converges at second order to the one obtained by
  integrating continuity in physical coordinates (derivatives at fixed z, integration in z by Gauss
  quadrature), an independent route to the sigma-coordinate formula;
* the pressure is hydrostatic.
"""
import numpy as np
import pytest

from paper_2601_04826_gb300 import inputs

G = 9.81


def rect(oracle, n):
    return oracle.Mesh.rect(n, n, 0.0, 1.0, 0.0, 1.0, bc=(0, 0, 0, 0))


def gl01(K):
    x, w = np.polynomial.legendre.leggauss(K)
    return 0.5 * (1.0 + x), 0.5 * w


def test_profile_is_the_moment_expansion(oracle):
    level, n = 3, 12
    Q = inputs.random_moments_2d(n, n, level, seed=2)
    zeta, wq = gl01(8)
    out = oracle.lift3d(oracle.Model(level, 2, g=G), rect(oracle, n), Q, zeta)
    h = Q[0]
    al = np.stack([Q[inputs.idx_alpha(level, 2, k)] / h for k in range(level + 1)])
    be = np.stack([Q[inputs.idx_beta(level, k)] / h for k in range(level + 1)])
    for j, z in enumerate(zeta):
        np.testing.assert_allclose(out[0, j], np.polynomial.legendre.legval(1.0 - 2.0 * z, al), rtol=1e-12,
                                   atol=1e-14)
        np.testing.assert_allclose(out[1, j], np.polynomial.legendre.legval(1.0 - 2.0 * z, be), rtol=1e-12,
                                   atol=1e-14)
    np.testing.assert_allclose(np.tensordot(wq, out[0], 1), al[0], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(np.tensordot(wq, out[1], 1), be[0], rtol=1e-12, atol=1e-14)


def test_no_penetration_at_the_bed(oracle):
    level, n = 2, 16
    Q = inputs.random_moments_2d(n, n, level, seed=3)
    X, Y = inputs.centers_2d(n, n)
    c1, c2 = 0.3, -0.2
    bed = (0.05 + c1 * X + c2 * Y).reshape(-1)
    out = oracle.lift3d(oracle.Model(level, 2, g=G), rect(oracle, n), Q, np.array([0.0, 0.5]), bed=bed)
    inner = np.zeros((n, n), dtype=bool)
    inner[1:-1, 1:-1] = True
    inner = inner.reshape(-1)
    w0 = c1 * out[0, 0] + c2 * out[1, 0]
    np.testing.assert_allclose(out[2, 0][inner], w0[inner], rtol=1e-11, atol=1e-13)


def test_swe_surface_velocity_matches_the_paper(oracle):
    n = 20
    X, Y = inputs.centers_2d(n, n)
    h = 1.0 + 0.3 * X - 0.2 * Y
    u = 0.4 - 0.5 * X + 0.25 * Y
    v = -0.1 + 0.2 * X + 0.6 * Y
    Q = np.stack([h, h * u, h * v]).reshape(3, -1)
    out = oracle.lift3d(oracle.Model(0, 2, g=G), rect(oracle, n), Q, np.array([1.0]))
    w_paper = -h * (-0.5) - h * 0.6
    inner = np.zeros((n, n), dtype=bool)
    inner[1:-1, 1:-1] = True
    np.testing.assert_allclose(out[2, 0].reshape(n, n)[inner], w_paper[inner], rtol=1e-11, atol=1e-13)


def _smooth_fields():
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    tp = 2 * sp.pi
    h = 1 + sp.Rational(1, 5) * sp.sin(tp * x) * sp.cos(tp * y)
    b = sp.Rational(1, 10) * sp.cos(tp * x) * sp.sin(tp * y)
    al = [sp.Rational(3, 10) * sp.cos(tp * y), sp.Rational(1, 10) * sp.sin(tp * x), sp.Rational(1, 20) * sp.cos(tp * (x + y))]
    be = [sp.Rational(1, 5) * sp.sin(tp * x), -sp.Rational(1, 10) * sp.cos(tp * x), sp.Rational(1, 25) * sp.sin(tp * (x - y))]
    zeta = (z - b) / h
    phi = [sp.Integer(1), 1 - 2 * zeta, 6 * zeta**2 - 6 * zeta + 1]  # P_k(1 - 2 zeta), k = 0, 1, 2
    u = sum(a * p for a, p in zip(al, phi))
    v = sum(c * p for c, p in zip(be, phi))
    div = sp.diff(u, x) + sp.diff(v, y)  # horizontal derivatives at fixed z
    f = {k: sp.lambdify((x, y), e, "numpy") for k, e in (("h", h), ("b", b))}
    f["al"] = [sp.lambdify((x, y), e, "numpy") for e in al]
    f["be"] = [sp.lambdify((x, y), e, "numpy") for e in be]
    f["div"] = sp.lambdify((x, y, z), div, "numpy")
    f["ub"] = sp.lambdify((x, y), u.subs(z, b) * sp.diff(b, x) + v.subs(z, b) * sp.diff(b, y), "numpy")
    return f


def _w_by_continuity(f, X, Y, zeta):
    """w(z) = u.grad b at the bed minus the integral of the horizontal divergence from b to z."""
    h, b = f["h"](X, Y), f["b"](X, Y)
    zq, wq = gl01(8)  # the integrand is a polynomial of degree 2 in z: exact
    out = np.empty((len(zeta),) + X.shape)
    for j, zt in enumerate(zeta):
        top = b + zt * h
        acc = np.zeros_like(X)
        for s, w in zip(zq, wq):
            acc += w * f["div"](X, Y, b + s * (top - b))
        out[j] = f["ub"](X, Y) - (top - b) * acc
    return out


def test_vertical_velocity_converges_to_continuity(oracle):
    f = _smooth_fields()
    level, zeta = 2, np.array([0.0, 0.3, 0.7, 1.0])
    errs = []
    for n in (16, 32, 64):
        X, Y = inputs.centers_2d(n, n)
        h = f["h"](X, Y)
        Q = np.zeros((inputs.nvars(level, 2), n * n))
        Q[0] = h.reshape(-1)
        for k in range(level + 1):
            Q[inputs.idx_alpha(level, 2, k)] = (h * f["al"][k](X, Y)).reshape(-1)
            Q[inputs.idx_beta(level, k)] = (h * np.broadcast_to(f["be"][k](X, Y), X.shape)).reshape(-1)
        mesh = oracle.Mesh.rect(n, n, 0.0, 1.0, 0.0, 1.0, bc=(0, 0, 0, 0))
        out = oracle.lift3d(oracle.Model(level, 2, g=G), mesh, Q, zeta, bed=f["b"](X, Y).reshape(-1))
        ref = _w_by_continuity(f, X, Y, zeta)
        inner = (slice(None), slice(2, -2), slice(2, -2))
        errs.append(np.max(np.abs(out[2].reshape(len(zeta), n, n)[inner] - ref[inner])))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)
    assert errs[-1] < 5e-3


def test_hydrostatic_pressure(oracle):
    level, n = 1, 6
    Q = inputs.random_moments_2d(n, n, level, seed=1)
    zeta = np.array([0.0, 0.25, 1.0])
    out = oracle.lift3d(oracle.Model(level, 2, g=G), rect(oracle, n), Q, zeta)
    for j, zt in enumerate(zeta):
        np.testing.assert_allclose(out[3, j], G * Q[0] * (1.0 - zt), rtol=1e-15)

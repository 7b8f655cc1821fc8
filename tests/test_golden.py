"""Pins of the oracle against expressions the paper prints (text fixtures under tests/golden/, each
citing its passage): the 2D shallow-water eigenvalues, the flux of the 2D shallow moment equations at
levels 1-4, and the flux and nonconservative matrix of the 1D VAM model.  The fixtures are evaluated
with SymPy at seeded states; the basis integrals A_ijk, M_kk are integrated exactly here, so nothing
on the expected side comes from the oracle."""
import os
import re

import numpy as np
import pytest

sp = pytest.importorskip("sympy")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
G = 9.81


def read_fixture(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, expr = line.split(":", 1)
        out[key.strip()] = expr.strip()
    return out


def test_swe_eigenvalues_as_printed(oracle):
    fx = read_fixture("swe_eigenvalues_2d.txt")
    h, hun, n2, g = sp.symbols("h hun n2 g", positive=True)
    lams = [sp.lambdify((h, hun, n2, g), sp.sympify(fx[k], locals={"h": h, "hun": hun, "n2": n2, "g": g}))
            for k in ("lambda0", "lambda1", "lambda2")]
    md = oracle.Model(0, 2, g=G)
    rng = np.random.default_rng(11)
    for _ in range(20):
        q = np.array([rng.uniform(0.1, 3.0), rng.normal(0, 1.0), rng.normal(0, 1.0)])
        nx, ny = rng.normal(size=2) * rng.uniform(0.3, 2.0)  # also non-unit normals
        J = np.zeros((3, 3))
        for c in range(3):
            d = 1e-6 * max(1.0, abs(q[c]))
            qp, qm = q.copy(), q.copy()
            qp[c] += d
            qm[c] -= d
            J[:, c] = (md.flux(qp, nx, ny) - md.flux(qm, nx, ny)) / (2 * d)
        got = np.sort(np.linalg.eigvals(J + md.nc_matrix(q, nx, ny)).real)
        want = np.sort([float(f(q[0], q[1] * nx + q[2] * ny, nx * nx + ny * ny, G)) for f in lams])
        np.testing.assert_allclose(got, want, rtol=1e-7, atol=1e-7)


def basis_integrals(N):
    z = sp.symbols("z")
    phi = [sp.legendre(k, 1 - 2 * z) for k in range(N + 1)]
    A = [[[sp.integrate(sp.expand(phi[i] * phi[j] * phi[k]), (z, 0, 1)) for k in range(N + 1)] for j in range(N + 1)]
         for i in range(N + 1)]
    M = [sp.integrate(sp.expand(phi[k] ** 2), (z, 0, 1)) for k in range(N + 1)]
    return A, M


def printed_row(expr, h, a, b, A, M, N, k, g):
    """Evaluates one row expression of the SME flux fixture at numbers (sum_ij expands over i, j)."""
    m = re.match(r"sum_ij\((.*)\)\s*/\s*M\[k\](.*)$", expr)
    env = {"h": h, "a": a, "b": b, "A": A, "M": M, "g": g, "k": k, "delta_k0": 1.0 if k == 0 else 0.0}
    if not m:
        return float(eval(expr, {"__builtins__": {}}, env))
    inner, rest = m.group(1), m.group(2)
    s = 0.0
    for i in range(N + 1):
        for j in range(N + 1):
            s += float(eval(inner, {"__builtins__": {}}, dict(env, i=i, j=j)))
    s /= float(M[k])
    if rest.strip():
        s += float(eval("0" + rest, {"__builtins__": {}}, env))
    return s


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_sme_flux_as_printed(oracle, N):
    fx = read_fixture("sme_flux_2d.txt")
    A, M = basis_integrals(N)
    md = oracle.Model(N, 2, g=G)
    rng = np.random.default_rng(N)
    for _ in range(5):
        h = rng.uniform(0.2, 2.0)
        a = rng.normal(0, 0.5, N + 1)
        b = rng.normal(0, 0.5, N + 1)
        q = np.zeros(md.nv)
        q[0] = h
        for k in range(N + 1):
            q[md.index_alpha(k)] = h * a[k]
            q[md.index_beta(k)] = h * b[k]
        for d, (nx, ny) in (("x", (1.0, 0.0)), ("y", (0.0, 1.0))):
            F = md.flux(q, nx, ny)
            want = np.zeros(md.nv)
            want[0] = printed_row(fx[f"F{d}_h"], h, a, b, A, M, N, 0, G)
            for k in range(N + 1):
                want[md.index_alpha(k)] = printed_row(fx[f"F{d}_alpha_k"], h, a, b, A, M, N, k, G)
                want[md.index_beta(k)] = printed_row(fx[f"F{d}_beta_k"], h, a, b, A, M, N, k, G)
            np.testing.assert_allclose(F, want, rtol=1e-12, atol=1e-12)


def test_vam_flux_and_nc_as_printed():
    from oracle import vam

    fx = read_fixture("vam_flux_nc.txt")
    sym = sp.symbols("h u0 u1 w0 w1 bx g")
    env = dict(zip(["h", "u0", "u1", "w0", "w1", "bx", "g"], sym))
    w2 = sp.sympify(fx["w2"], locals=env)
    env["w2"] = w2
    F = [sp.lambdify(sym, sp.sympify(fx[f"F{r}"], locals=env)) for r in range(5)]
    nc = {(1, 0): fx["NC[1][0]"], (2, 2): fx["NC[2][2]"], (4, 2): fx["NC[4][2]"]}
    nc = {rc: sp.lambdify(sym, sp.sympify(e, locals=env)) for rc, e in nc.items()}
    rng = np.random.default_rng(5)
    for _ in range(20):
        h = rng.uniform(0.3, 2.0)
        u0, u1, w0, w1, bx = rng.normal(0, 0.5, 5)
        Q = np.array([[h], [h * u0], [h * u1], [h * w0], [h * w1]])
        args = (h, u0, u1, w0, w1, bx, G)
        # the oracle writes the gravity g h dh/dx as the flux g h^2/2 (equal on any straight path)
        got_F = vam.flux(Q, G, bx)[:, 0] - np.array([0.0, 0.5 * G * h * h, 0.0, 0.0, 0.0])
        np.testing.assert_allclose(got_F, [float(f(*args)) for f in F], rtol=1e-13, atol=1e-13)
        dQ = rng.normal(size=(5, 1))
        got_nc = vam.nc_times(Q, dQ, bx)[:, 0]
        got_nc[1] += G * h * dQ[0, 0]
        want_nc = np.zeros(5)
        for (r, c), f in nc.items():
            want_nc[r] += float(f(*args)) * dQ[c, 0]
        np.testing.assert_allclose(got_nc, want_nc, rtol=1e-13, atol=1e-13)

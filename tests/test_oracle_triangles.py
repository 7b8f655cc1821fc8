"""Pins of the oracle's triangle-mesh path (face frames, geometry, neighbours) against things that
do not come from the oracle:

* a planar Stoker dam break on jittered Delaunay meshes converges to the 1D closed form (a wrong
  normal, edge length, area or neighbour breaks convergence);
* a lake at rest over a dyadic bathymetry with a dry island stays at rest bitwise;
* rotating the mesh by 90 degrees (exact in floating point) rotates the solution: the face-frame
  rotation and its inverse are consistent.
"""
import numpy as np
from scipy.optimize import brentq

from paper_2601_04826_gb300 import inputs

G = 9.81


def stoker_h(x, t, x0, hl, hr):
    cl = np.sqrt(G * hl)

    def f(hm):
        return 2 * (cl - np.sqrt(G * hm)) - (hm - hr) * np.sqrt(G * (hm + hr) / (2 * hm * hr))

    hm = brentq(f, hr, hl)
    um = 2 * (cl - np.sqrt(G * hm))
    S = hm * um / (hm - hr)
    xi = (x - x0) / t
    h = np.where(xi <= -cl, hl, (2 * cl - xi) ** 2 / (9 * G))
    h = np.where(xi >= um - np.sqrt(G * hm), hm, h)
    return np.where(xi >= S, hr, h)


def run_to(oracle, md, mesh, Q, T, bed=None):
    t, n = 0.0, 0
    while t < T - 1e-14:
        dt = min(oracle.cfl_dt(md, mesh, Q, 0.45), T - t)
        assert np.isfinite(dt) and dt > 0.0 and n < 5000
        Q, _ = oracle.step(md, mesh, Q, 1, dt=dt, bed=bed)
        t += dt
        n += 1
    return Q


def areas(verts, tris):
    p = verts[tris]
    return 0.5 * np.abs((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                        - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))


def test_planar_stoker_on_triangles_converges(oracle):
    # dam at x = 0 on [-1, 1]^2; by T = 0.15 no wave has reached the walls at x = +-1
    T, hl, hr = 0.15, 2.0, 1.0
    md = oracle.Model(1, 2, g=G)
    errs = []
    for n_side in (21, 41, 81):
        verts, tris = inputs.jittered_delaunay(n_side, seed=n_side)
        c = inputs.tri_centroids(verts, tris)
        Q = np.zeros((inputs.nvars(1, 2), len(tris)))
        Q[0] = np.where(c[:, 0] < 0.0, hl, hr)
        mesh = oracle.Mesh.triangles(verts, tris, bc=1)
        Q = run_to(oracle, md, mesh, Q, T)
        A = areas(verts, tris)
        errs.append(np.sum(A * np.abs(Q[0] - stoker_h(c[:, 0], T, 0.0, hl, hr))))
        # y-uniform problem: the transverse momentum stays small against the normal one
        assert np.sum(A * np.abs(Q[2])) < 0.1 * np.sum(A * np.abs(Q[1]))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates >= 0.5), (errs, rates)


def test_lake_at_rest_on_triangles_bitwise(oracle):
    verts, tris = inputs.jittered_delaunay(24, seed=9)
    c = inputs.tri_centroids(verts, tris)
    b = 0.3 * np.sin(np.pi * c[:, 0]) * np.cos(np.pi * c[:, 1]) + 0.9 * np.exp(-(c[:, 0] ** 2 + c[:, 1] ** 2) / 0.02)
    b = np.round(b * 65536.0) / 65536.0
    level = 2
    Q = np.zeros((inputs.nvars(level, 2), len(tris)))
    Q[0] = np.maximum(0.75 - b, 0.0)
    assert np.any(Q[0] == 0.0) and np.any(Q[0] > 0.0)
    md = oracle.Model(level, 2, g=G, friction=1, C=0.1, nu=0.01)
    mesh = oracle.Mesh.triangles(verts, tris, bc=1)
    R, _ = oracle.step(md, mesh, Q, 200, bed=b)
    np.testing.assert_array_equal(R[0], Q[0])
    np.testing.assert_array_equal(R[1:], 0.0)


def test_quarter_turn_rotates_the_solution(oracle):
    level = 2
    verts, tris = inputs.jittered_delaunay(18, seed=4)
    rng = np.random.default_rng(1)
    Q = np.zeros((inputs.nvars(level, 2), len(tris)))
    c = inputs.tri_centroids(verts, tris)
    Q[0] = 1.0 + 0.3 * np.exp(-((c[:, 0] - 0.2) ** 2 + (c[:, 1] + 0.1) ** 2) / 0.05)
    for v in range(1, Q.shape[0]):
        Q[v] = Q[0] * rng.uniform(-0.2, 0.2, len(tris))
    rot = np.stack([-verts[:, 1], verts[:, 0]], axis=1)  # (x, y) -> (-y, x), exact
    md = oracle.Model(level, 2, g=G, friction=1, C=0.1, nu=0.01)
    ia = [inputs.idx_alpha(level, 2, k) for k in range(level + 1)]
    ib = [inputs.idx_beta(level, k) for k in range(level + 1)]
    Qr = Q.copy()
    for k in range(level + 1):  # vectors (a, b) -> (-b, a)
        Qr[ia[k]] = -Q[ib[k]]
        Qr[ib[k]] = Q[ia[k]]
    R, _ = oracle.step(md, oracle.Mesh.triangles(verts, tris, bc=1), Q, 10, dt=2e-3)
    Rr, _ = oracle.step(md, oracle.Mesh.triangles(rot, tris, bc=1), Qr, 10, dt=2e-3)
    back = Rr.copy()
    for k in range(level + 1):
        back[ia[k]] = Rr[ib[k]]
        back[ib[k]] = -Rr[ia[k]]
    np.testing.assert_allclose(back, R, rtol=1e-11, atol=1e-13)

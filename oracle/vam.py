"""FP64 oracle of the non-hydrostatic VAM predictor-corrector in 1D -- TEST INFRASTRUCTURE ONLY.

The paper's vertically averaged momentum model (Sec. "Unsteady Vertically Averaged Momentum
Equations in 1D", with the splitting Eq. (PDE-hyperbolic) - Eq. (PDE-source)) over a bed b(x):

    Q = (h, h u0, h u1, h w0, h w1),  w2 = -(w0 + w1) + (u0 + u1) b_x
    F = (h u0, h u0^2 + h u1^2 / 3 + g h^2 / 2, 2 h u0 u1, h u0 w0 + h u1 w1 / 3,
         h u0 w1 + u1 (h w0 + 2/5 h w2))
    nonconservative product B(Q) dQ/dx: rows h u1: -u0 d(h u1)/dx;  h w1: (w2/5 - w0) d(h u1)/dx
    (the g h dh/dx of row h u0 is written as the flux g h^2 / 2, and the bed force g h b_x comes from
    the hydrostatic reconstruction);
    pressure part S(p) = (0, d(h p0)/dx + 2 p1 b_x, d(h p1)/dx - (3 p0 - p1) dh/dx - 6 (p0 - p1) b_x,
                          -2 p1, 6 (p0 - p1)),
    constraints R0 = h du0/dx + d(h u1)/dx / 3 + u1 dh/dx / 3 + 2 (w0 - u0 b_x) = 0,
                R1 = h du0/dx + u1 dh/dx + 2 (u1 b_x - w1) = 0.

One step (reading R19):
  1. predictor: hydrostatic reconstruction at every face (b_f = max(b_L, b_R), h* = max(0, h + b - b_f),
     velocities kept), the conservative flux Phi = (F(L*) + F(R*))/2 - s_f (R* - L*)/2 and the path
     integral Btilde (R* - L*) by 3-point Gauss-Legendre on the straight segment; cell i takes
     Q* = Q - dt/dx [(Phi - P(h*_i) e1 + Btilde dQ/2)_{i+1/2} - (Phi - P(h*_i) e1 - Btilde dQ/2)_{i-1/2}],
     P(h) = g h^2 / 2, s_f = max of s = |u0| + sqrt(g h* + u1^2) + |u1| on both reconstructed states;
  2. corrector: p0, p1 per cell such that Q** = Q* - dt S(p) satisfies R0(Q**) = R1(Q**) = 0, with
     central differences (q_{i+1} - q_{i-1}) / (2 dx) and ghost cells (walls: u0, u1 and their
     momenta change sign; h, w0, w1, p0, p1 and b mirror); the system is linear in p: its matrix is
     assembled column by column from R(e_j) - R(0) and solved densely;
  3. Q^{n+1} = Q**.
b_x is the central difference of b per cell (bed ghosts copy the boundary cell); in a flux the cell's
own b_x is used, along a face path the mean of the two cells' (a wall ghost's b_x changes sign, as a
slope does under reflection).  dt = cfl dx / max_i s_i from Q^n, or fixed.  h must stay positive
(no dry states); a reconstructed face depth may reach 0, where velocities are taken as 0.
"""
from __future__ import annotations

import numpy as np

SQ = np.array([0.5 - np.sqrt(15.0) / 10.0, 0.5, 0.5 + np.sqrt(15.0) / 10.0])
WQ = np.array([5.0, 8.0, 5.0]) / 18.0
ODD = np.array([1.0, -1.0, -1.0, 1.0, 1.0])  # wall ghost: horizontal momenta change sign


def prim(Q, bx=0.0):
    h = Q[0]
    ih = np.divide(1.0, h, out=np.zeros_like(h), where=h > 0.0)
    u0, u1, w0, w1 = Q[1] * ih, Q[2] * ih, Q[3] * ih, Q[4] * ih
    return h, u0, u1, w0, w1, -(w0 + w1) + (u0 + u1) * bx


def flux(Q, g, bx=0.0):
    h, u0, u1, w0, w1, w2 = prim(Q, bx)
    return np.stack([h * u0, h * u0 * u0 + h * u1 * u1 / 3.0 + 0.5 * g * h * h, 2.0 * h * u0 * u1,
                     h * u0 * w0 + h * u1 * w1 / 3.0, h * u0 * w1 + u1 * (h * w0 + 0.4 * h * w2)])


def nc_times(Q, dQ, bx=0.0):
    """B(Q) dQ for states Q [5, n] and differences dQ [5, n] (the gravity part is in the flux)."""
    h, u0, u1, w0, w1, w2 = prim(Q, bx)
    out = np.zeros_like(dQ)
    out[2] = -u0 * dQ[2]
    out[4] = (w2 / 5.0 - w0) * dQ[2]
    return out


def wavespeed(Q, g):
    h, u0, u1, *_ = prim(Q)
    return np.abs(u0) + np.sqrt(g * h + u1 * u1) + np.abs(u1)


def ghosted(Q, bc):
    """State with one ghost cell at each end: bc = (left, right), 1 wall, 0 transmissive."""
    gl = Q[:, :1] * (ODD[:, None] if bc[0] == 1 else 1.0)
    gr = Q[:, -1:] * (ODD[:, None] if bc[1] == 1 else 1.0)
    return np.concatenate([gl, Q, gr], axis=1)


def bed_slope(b, dx, bc):
    """b_x per cell and per ghost: central differences with copied bed ghosts; a wall ghost's slope
    changes sign."""
    bx = diff(b, dx, bc, False)
    sl = -1.0 if bc[0] == 1 else 1.0
    sr = -1.0 if bc[1] == 1 else 1.0
    return bx, np.concatenate([[sl * bx[0]], bx, [sr * bx[-1]]])


def predictor(Q, dt, dx, g, bc, b=None):
    n = Q.shape[1]
    b = np.zeros(n) if b is None else np.asarray(b, dtype=np.float64)
    _, bxg = bed_slope(b, dx, bc)
    Qg = ghosted(Q, bc)
    bg = np.concatenate([[b[0]], b, [b[-1]]])
    L, R = Qg[:, :-1], Qg[:, 1:]  # faces i-1/2 for i = 0..n
    bL, bR, bxL, bxR = bg[:-1], bg[1:], bxg[:-1], bxg[1:]
    bf = np.maximum(bL, bR)
    hLs = np.maximum(0.0, L[0] + bL - bf)
    hRs = np.maximum(0.0, R[0] + bR - bf)
    Ls = L * np.divide(hLs, L[0], out=np.zeros_like(hLs), where=L[0] > 0.0)
    Rs = R * np.divide(hRs, R[0], out=np.zeros_like(hRs), where=R[0] > 0.0)
    Ls[0], Rs[0] = hLs, hRs
    dQ = Rs - Ls
    bxf = 0.5 * (bxL + bxR)
    Bt = sum(w * nc_times(Ls + s * dQ, dQ, bxf) for s, w in zip(SQ, WQ))
    sf = np.maximum(wavespeed(Ls, g), wavespeed(Rs, g))
    Phi = 0.5 * (flux(Ls, g, bxL) + flux(Rs, g, bxR)) - 0.5 * sf * dQ
    Gm = Phi + 0.5 * Bt  # to the left cell of the face (its right face)
    Gm[1] -= 0.5 * g * hLs * hLs
    Gp = Phi - 0.5 * Bt  # to the right cell (its left face)
    Gp[1] -= 0.5 * g * hRs * hRs
    return Q - dt / dx * (Gm[:, 1:] - Gp[:, :-1])


def diff(x, dx, bc, odd):
    """Central difference with mirrored (odd: sign-changed at walls) ghost values."""
    sl = -1.0 if (odd and bc[0] == 1) else 1.0
    sr = -1.0 if (odd and bc[1] == 1) else 1.0
    xg = np.concatenate([[sl * x[0]], x, [sr * x[-1]]])
    return (xg[2:] - xg[:-2]) / (2.0 * dx)


def corrected(Qs, p0, p1, dt, dx, bc, bx=0.0):
    """Q** = Q* - dt S(p)."""
    h = Qs[0]
    dh = diff(h, dx, bc, False)
    Q = Qs.copy()
    Q[1] = Qs[1] - dt * (diff(h * p0, dx, bc, False) + 2.0 * p1 * bx)
    Q[2] = Qs[2] - dt * (diff(h * p1, dx, bc, False) - (3.0 * p0 - p1) * dh - 6.0 * (p0 - p1) * bx)
    Q[3] = Qs[3] + dt * 2.0 * p1
    Q[4] = Qs[4] - dt * 6.0 * (p0 - p1)
    return Q


def residual(Qs, p, dt, dx, bc, bx=0.0):
    """(R0, R1) of Q** = Q* - dt S(p), p = (p0_0, p1_0, p0_1, ...); interleaved like p."""
    p0, p1 = p[0::2], p[1::2]
    Q = corrected(Qs, p0, p1, dt, dx, bc, bx)
    h, u0, u1, w0, w1, _ = prim(Q)
    dh = diff(h, dx, bc, False)
    du0 = diff(u0, dx, bc, True)
    R0 = h * du0 + diff(Q[2], dx, bc, True) / 3.0 + u1 * dh / 3.0 + 2.0 * (w0 - u0 * bx)
    R1 = h * du0 + u1 * dh + 2.0 * (u1 * bx - w1)
    out = np.empty(2 * len(h))
    out[0::2], out[1::2] = R0, R1
    return out


def corrector(Qs, dt, dx, bc, b=None):
    """Pressure p solving the linear constraints, and Q**."""
    bx = 0.0 if b is None else bed_slope(np.asarray(b, dtype=np.float64), dx, bc)[0]
    n2 = 2 * Qs.shape[1]
    r0 = residual(Qs, np.zeros(n2), dt, dx, bc, bx)
    J = np.empty((n2, n2))
    for j in range(n2):
        e = np.zeros(n2)
        e[j] = 1.0
        J[:, j] = residual(Qs, e, dt, dx, bc, bx) - r0
    p = np.linalg.solve(J, -r0)
    return corrected(Qs, p[0::2], p[1::2], dt, dx, bc, bx), p


def step(Q, nsteps, dx, g=9.81, bc=(1, 1), cfl=0.45, dt=0.0, b=None):
    """nsteps predictor-corrector steps over the bed b (None: flat); returns (Q, t advanced, last pressure)."""
    Q = np.array(Q, dtype=np.float64)
    t, p = 0.0, None
    for _ in range(nsteps):
        d = dt if dt > 0.0 else cfl * dx / wavespeed(Q, g).max()
        Qs = predictor(Q, d, dx, g, bc, b)
        Q, p = corrector(Qs, d, dx, bc, b)
        t += d
    return Q, t, p


def jacobian_eigenvalues(q, g, bx=0.0):
    """Eigenvalues of dF/dQ + B(Q) at one state (for the wave-speed bound)."""
    q = np.asarray(q, dtype=np.float64)
    J = np.zeros((5, 5))
    eps = 1e-7
    for j in range(5):
        e = np.zeros(5)
        e[j] = eps * max(1.0, abs(q[j]))
        J[:, j] = (flux((q + e)[:, None], g, bx)[:, 0] - flux((q - e)[:, None], g, bx)[:, 0]) / (2.0 * e[j])
        J[:, j] += nc_times(q[:, None], (e / e[j])[:, None], bx)[:, 0]
    return np.linalg.eigvals(J)

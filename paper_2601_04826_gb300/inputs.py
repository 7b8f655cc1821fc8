"""Seeded synthetic inputs shared by the tests, bench.py and smoke().

This module only builds initial states, bathymetries and meshes from seeds; it
holds none of the finite-volume method's arithmetic, so the GPU library and the
CPU oracle can both be fed from it.  Every array is float64; a caller that runs
the FP32 path casts once and gives the oracle the same rounded values.

Variable order (the library's and the oracle's):
  1D: (h, h alpha_0, ..., h alpha_N)
  2D: (h, h alpha_0, h beta_0, h alpha_1..h alpha_N, h beta_1..h beta_N)
"""
from __future__ import annotations

import numpy as np


def nvars(level: int, dim: int) -> int:
    return 1 + (level + 1) * (1 if dim == 1 else 2)


def idx_alpha(level: int, dim: int, k: int) -> int:
    if dim == 1:
        return 1 + k
    return 1 if k == 0 else 2 + k


def idx_beta(level: int, k: int) -> int:
    return 2 if k == 0 else 2 + level + k


# ----------------------------------------------------------------------------- 1D

def centers_1d(nx: int, x0: float, x1: float) -> np.ndarray:
    dx = (x1 - x0) / nx
    return x0 + (np.arange(nx) + 0.5) * dx


def dambreak_1d(nx=2000, x0=0.0, x1=10.0, h_left=2.0, h_right=1.0, x_dam=5.0, level=1,
                u=0.0, alpha=None) -> np.ndarray:
    """Dam break at rest: h = h_left for x < x_dam else h_right; optional uniform u and moments."""
    x = centers_1d(nx, x0, x1)
    Q = np.zeros((nvars(level, 1), nx))
    Q[0] = np.where(x < x_dam, h_left, h_right)
    Q[1] = Q[0] * u
    if alpha is not None:
        for k, a in enumerate(alpha, start=1):
            Q[idx_alpha(level, 1, k)] = Q[0] * a
    return Q


# ----------------------------------------------------------------------------- 2D structured

def centers_2d(nx: int, ny: int, x0=0.0, x1=1.0, y0=0.0, y1=1.0):
    xc = x0 + (np.arange(nx) + 0.5) * (x1 - x0) / nx
    yc = y0 + (np.arange(ny) + 0.5) * (y1 - y0) / ny
    X, Y = np.meshgrid(xc, yc, indexing="xy")  # [ny, nx], cell (i, j) at [j, i]
    return X, Y


def fourier_bathymetry(X, Y, rng, modes=8, amplitude=0.2) -> np.ndarray:
    """b = amplitude * sum_m a_m cos(2 pi k_m . x + theta_m), k_m in {1..4}^2, sum |a_m| = 1."""
    k = rng.integers(1, 5, size=(modes, 2))
    a = rng.uniform(-1.0, 1.0, size=modes)
    a /= np.abs(a).sum()
    th = rng.uniform(0.0, 2.0 * np.pi, size=modes)
    b = np.zeros_like(X)
    for m in range(modes):
        b += a[m] * np.cos(2.0 * np.pi * (k[m, 0] * X + k[m, 1] * Y) + th[m])
    return amplitude * b


def gaussian_bump_2d(nx, ny, level, seed=0, bathymetry=True, amp_range=(0.1, 0.5), sigma=0.05,
                     eta0=1.0, center_range=(0.3, 0.7), x0=0.0, x1=1.0, y0=0.0, y1=1.0,
                     moments=None):
    """Gaussian surface bump on a lake of level eta0 over smooth random bathymetry.

    Returns (Q [nv, ny*nx], b [ny*nx]) with cell (i, j) at flat index j*nx + i.
    ``moments`` optionally sets uniform velocity moments {var_index: value_per_depth}.
    """
    rng = np.random.default_rng(seed)
    X, Y = centers_2d(nx, ny, x0, x1, y0, y1)
    b = fourier_bathymetry(X, Y, rng) if bathymetry else np.zeros_like(X)
    amp = rng.uniform(*amp_range)
    cx, cy = rng.uniform(*center_range, size=2)
    eta = eta0 + amp * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * sigma**2))
    h = np.maximum(eta - b, 0.0)
    Q = np.zeros((nvars(level, 2), ny * nx))
    Q[0] = h.reshape(-1)
    if moments:
        for v, a in moments.items():
            Q[v] = Q[0] * a
    return Q, b.reshape(-1)


def random_moments_2d(nx, ny, level, seed=0, h_range=(0.5, 1.5), vel=0.3, smooth=True):
    """Smooth random state with all velocity moments non-zero (flat bed)."""
    rng = np.random.default_rng(seed)
    X, Y = centers_2d(nx, ny)
    nv = nvars(level, 2)
    Q = np.zeros((nv, ny * nx))

    def field(scale):
        k = rng.integers(1, 4, size=(3, 2))
        th = rng.uniform(0, 2 * np.pi, size=3)
        a = rng.uniform(-1, 1, size=3)
        f = sum(a[i] * np.sin(2 * np.pi * (k[i, 0] * X + k[i, 1] * Y) + th[i]) for i in range(3))
        return scale * f / 3.0

    h = 0.5 * (h_range[0] + h_range[1]) + field(0.5 * (h_range[1] - h_range[0]))
    Q[0] = h.reshape(-1)
    for v in range(1, nv):
        Q[v] = (h * field(vel)).reshape(-1)
    return Q


def lake_at_rest_dyadic(nx, ny, level, seed=0, eta=0.75):
    """Lake at rest over a bathymetry of multiples of 2^-16 with a dry island.

    h = max(eta - b, 0) is exact in FP32 and FP64, so the surface is exactly flat.
    """
    rng = np.random.default_rng(seed)
    X, Y = centers_2d(nx, ny)
    b = 0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y) + 0.1 * rng.uniform(-1, 1, X.shape)
    island = np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / 0.01)
    b = b + 0.9 * island
    b = np.round(b * 65536.0) / 65536.0
    h = np.maximum(eta - b, 0.0)
    Q = np.zeros((nvars(level, 2), ny * nx))
    Q[0] = h.reshape(-1)
    return Q, b.reshape(-1)


# ----------------------------------------------------------------------------- triangles

def jittered_delaunay(n_side: int, seed=0, jitter=0.3, lo=-1.0, hi=1.0):
    """Jittered lattice of n_side^2 points on [lo,hi]^2 triangulated by Delaunay.

    Interior points move by up to ``jitter`` lattice spacings in x and y; boundary
    points move only along their edge and the corners stay put, so the hull is the
    square.  Returns (verts [nv, 2] float64, tris [nt, 3] int32, counter-clockwise).
    """
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    s = (hi - lo) / (n_side - 1)
    g = lo + s * np.arange(n_side)
    X, Y = np.meshgrid(g, g, indexing="xy")
    dx = rng.uniform(-jitter, jitter, X.shape) * s
    dy = rng.uniform(-jitter, jitter, X.shape) * s
    onx = np.zeros_like(X, dtype=bool)
    ony = np.zeros_like(X, dtype=bool)
    onx[:, [0, -1]] = True
    ony[[0, -1], :] = True
    dx[onx] = 0.0
    dy[ony] = 0.0
    pts = np.stack([(X + dx).reshape(-1), (Y + dy).reshape(-1)], axis=1)
    tri = Delaunay(pts)
    t = tri.simplices.astype(np.int32)
    p = pts[t]
    area2 = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1])
    neg = area2 < 0
    t[neg] = t[neg][:, [0, 2, 1]]
    keep = np.abs(area2) > 1e-14 * s * s
    return pts, np.ascontiguousarray(t[keep])


def tri_centroids(verts, tris):
    return verts[tris].mean(axis=1)


def circular_dam_tri(verts, tris, level, radius=0.2, h_in=1.5, h_out=0.0):
    """Circular dam break on triangles: h = h_in inside r < radius, h_out outside, at rest."""
    c = tri_centroids(verts, tris)
    r = np.hypot(c[:, 0], c[:, 1])
    Q = np.zeros((nvars(level, 2), len(tris)))
    Q[0] = np.where(r < radius, h_in, h_out)
    return Q


# ----------------------------------------------------------------------------- ensemble

def ensemble_members(n_members=512, seed=0, side_lo=64, side_hi=512, mu=-2.0, sigma=0.5):
    """Member sides ~ U{side_lo..side_hi}, slip coefficients ~ logNormal(mu, sigma), bump seeds."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=n_members)
    lam = rng.lognormal(mu, sigma, size=n_members)
    seeds = rng.integers(0, 2**31 - 1, size=n_members)
    return sides, lam, seeds


def ensemble_state(sides, seeds, level, amp_range=(0.1, 0.5), sigma=0.05):
    """Concatenated initial states of square members: base depth 1, flat bed, at rest, with a
    seeded Gaussian bump per member.  Returns (Q [nv, sum side^2], offsets [nmembers + 1])."""
    offs = np.concatenate([[0], np.cumsum(np.asarray(sides, dtype=np.int64) ** 2)])
    Q = np.zeros((nvars(level, 2), offs[-1]))
    for m, (s, sd) in enumerate(zip(sides, seeds)):
        Qm, _ = gaussian_bump_2d(int(s), int(s), level, seed=int(sd), bathymetry=False, amp_range=amp_range,
                                 sigma=sigma)
        Q[:, offs[m]:offs[m + 1]] = Qm
    return Q, offs

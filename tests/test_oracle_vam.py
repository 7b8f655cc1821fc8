"""Pins of the oracle's VAM predictor-corrector (reading R19) against physics that the model must
reproduce, not against itself:

* linear dispersion: a small standing wave in a closed basin oscillates with the phase speed of
  linear water-wave theory, c^2 = g tanh(kH)/k (Airy), to within 0.6 % up to kH = 2, and with the
  model's own linear dispersion relation c^2/(gH) = (1 + K/12)/(1 + 5K/12 + K^2/144), K = (kH)^2,
  derived by hand from the linearised equations, to within 0.2 %; the hydrostatic limit is far off
  (c^2 = gH); long waves recover c^2 = gH;
* a lake at rest stays at rest bitwise; mass is conserved between walls; after every step the two
  constraints of the corrector hold; the wave-speed bound covers the spectrum of the hyperbolic part;
* mistakes planted in a copy of the oracle (a source sign, a dropped pressure term) break the
  dispersion pin.
"""
import importlib.util
import os
import sys

import numpy as np
import pytest

from oracle import vam

G, H = 9.81, 1.0
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def standing_wave_c2(mod, kH, N=100, amp=1e-3):
    """c^2/(gH) from the first zero crossing of h - H at the left wall (a quarter period)."""
    k = kH / H
    L = np.pi / k
    dx = L / N
    x = (np.arange(N) + 0.5) * dx
    Q = np.zeros((5, N))
    Q[0] = H + amp * np.cos(k * x)
    hs, ts, t = [Q[0, 0]], [0.0], 0.0
    for _ in range(20 * N):
        Q, dt, _ = mod.step(Q, 1, dx, g=G, bc=(1, 1))
        t += dt
        hs.append(Q[0, 0])
        ts.append(t)
        if Q[0, 0] < H or not np.isfinite(Q[0, 0]):
            break
    y0, y1 = hs[-2] - H, hs[-1] - H
    tz = ts[-2] + (ts[-1] - ts[-2]) * y0 / (y0 - y1)
    om = np.pi / (2.0 * tz)
    return (om / k) ** 2 / (G * H)


def vam_linear(kH):
    K = kH * kH
    return (1.0 + K / 12.0) / (1.0 + 5.0 * K / 12.0 + K * K / 144.0)


@pytest.mark.parametrize("kH", [0.5, 1.0, 2.0])
def test_dispersion_matches_linear_wave_theory(kH):
    c2 = standing_wave_c2(vam, kH)
    airy = np.tanh(kH) / kH
    assert abs(c2 - airy) < 6e-3 * airy, (c2, airy)
    assert abs(c2 - vam_linear(kH)) < 2e-3 * vam_linear(kH), (c2, vam_linear(kH))
    if kH >= 1.0:
        assert c2 < 0.8  # far from the hydrostatic c^2 = gH


def test_long_waves_are_hydrostatic():
    assert standing_wave_c2(vam, 0.1, N=60) == pytest.approx(1.0, abs=5e-3)


def test_lake_at_rest_bitwise():
    Q = np.zeros((5, 40))
    Q[0] = 0.8
    R, _, p = vam.step(Q, 20, 0.05)
    np.testing.assert_array_equal(R, Q)
    np.testing.assert_array_equal(p, 0.0)


def test_mass_and_constraints():
    n, dx = 64, 1.0 / 64
    x = (np.arange(n) + 0.5) * dx
    rng = np.random.default_rng(0)
    Q = np.zeros((5, n))
    Q[0] = 1.0 + 0.1 * np.exp(-((x - 0.4) ** 2) / 0.01)
    Q[1] = Q[0] * 0.05 * np.sin(2 * np.pi * x)
    Q[2] = Q[0] * 0.02 * rng.normal(size=n)
    m0 = Q[0].sum()
    for _ in range(10):
        d = 0.3 * dx / vam.wavespeed(Q, G).max()
        Qs = vam.predictor(Q, d, dx, G, (1, 1))
        Q, p = vam.corrector(Qs, d, dx, (1, 1))
        R = vam.residual(Qs, p, d, dx, (1, 1))
        assert np.abs(R).max() < 1e-9 * max(1.0, np.abs(p).max())
    assert abs(Q[0].sum() - m0) / m0 < 1e-13


def test_wavespeed_bounds_the_spectrum():
    rng = np.random.default_rng(3)
    for _ in range(200):
        h = rng.uniform(0.1, 2.0)
        q = np.array([h, *(h * rng.normal(0.0, 0.5, 4))])
        lam = vam.jacobian_eigenvalues(q, G)
        s = vam.wavespeed(q[:, None], G)[0]
        assert np.max(np.abs(lam.real)) <= s * (1 + 1e-6)


MUTANTS = {
    "w1_source_sign": ("Q[4] = Qs[4] - dt * 6.0 * (p0 - p1)", "Q[4] = Qs[4] + dt * 6.0 * (p0 - p1)"),
    "u1_pressure_gradient_dropped": ("diff(h * p1, dx, bc, False) - (3.0 * p0 - p1) * dh", "-(3.0 * p0 - p1) * dh"),
    "u0_pressure_sign": ("Q[1] = Qs[1] - dt * (diff(h * p0", "Q[1] = Qs[1] + dt * (diff(h * p0"),
    "w0_constraint_factor": ("u1 * dh / 3.0 + 2.0 * (w0 - u0 * bx)", "u1 * dh / 3.0 + (w0 - u0 * bx)"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_dispersion_pin_catches_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "vam.py")).read()
    assert src.count(old) == 1
    path = tmp_path / f"vam_{name}.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"vam_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    with np.errstate(all="ignore"):
        try:
            c2 = standing_wave_c2(mod, 1.0, N=60)
        except (np.linalg.LinAlgError, FloatingPointError, ValueError):
            return
    assert not abs(c2 - np.tanh(1.0)) < 6e-3 * np.tanh(1.0), c2


# ---- the bed terms (b_x in S, R0, R1 and w2) -----------------------------------------------------

def pressure_work_defect(mod, n, L=8.0, bed=True):
    """The pressure does no work on flows that satisfy the constraints: with the kinetic-energy
    weights (1, 1/3, 1, 1/3) of (u0, u1, w0, w1), the power of the force -S(p) equals the pairing of p
    with the constraints, sum u . W S(p) = -sum [p0 R1(u) + p1 (R0(u) - R1(u))] (derived from the
    equations by integration by parts, bed terms included).  Smooth, compactly supported fields; the
    discrete defect is the central differences' truncation error.  Returns |lhs + rhs| / |lhs|."""
    dx = L / n
    x = (np.arange(n) + 0.5) * dx
    h = 1.0 + 0.2 * np.sin(0.9 * x) + 0.1 * np.cos(2.1 * x)
    bx = 0.0
    b = 0.3 * np.cos(1.3 * x) + 0.1 * np.sin(0.7 * x) if bed else np.zeros(n)
    bump = lambda c, w: np.exp(-(((x - c) / w) ** 2))
    vel = [bump(3.0, 0.6) * np.sin(2.0 * x), bump(4.5, 0.7), bump(3.8, 0.5) * np.cos(x), bump(4.2, 0.6) * x]
    p0, p1 = bump(4.0, 0.8) * np.cos(1.5 * x), bump(3.6, 0.7) * (1.0 + x)
    bc = (1, 1)
    bx = mod.bed_slope(b, dx, bc)[0]
    Qs = np.stack([h] + [h * v for v in vel])
    dt = 1.0
    S = (Qs - mod.corrected(Qs, p0, p1, dt, dx, bc, bx)) / dt
    W = [1.0, 1.0 / 3.0, 1.0, 1.0 / 3.0]
    lhs = sum(W[k] * np.sum(vel[k] * S[1 + k]) for k in range(4))
    R = mod.residual(Qs, np.zeros(2 * n), dt, dx, bc, bx)
    R0, R1 = R[0::2], R[1::2]
    rhs = np.sum(p0 * R1 + p1 * (R0 - R1))
    return abs(lhs + rhs) / abs(lhs)


@pytest.mark.parametrize("bed", [False, True])
def test_pressure_does_no_work(bed):
    d1, d2 = pressure_work_defect(vam, 400, bed=bed), pressure_work_defect(vam, 800, bed=bed)
    assert d2 < 1e-3, (d1, d2)
    assert 3.0 < d1 / d2 < 5.0, (d1, d2)  # second-order truncation, no O(1) mismatch


def slope_stream_residual(mod, S=0.05, U=0.7, H=0.8, n=64):
    """A stream parallel to a uniformly sloping bed b = -S x (u0 = U, u1 = 0, w = u b_x = -U S)
    satisfies both constraints exactly; the interior cells' residual at p = 0 vanishes."""
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    b = -S * x
    Q = np.stack([np.full(n, H), np.full(n, H * U), np.zeros(n), np.full(n, -H * U * S), np.zeros(n)])
    bx = mod.bed_slope(b, dx, (0, 0))[0]
    R = mod.residual(Q, np.zeros(2 * n), 0.01, dx, (0, 0), bx)
    return np.abs(R[4:-4]).max() / (U * S)


def test_slope_parallel_stream_satisfies_constraints():
    assert slope_stream_residual(vam) < 1e-12
    h, u0, u1, w0, w1, w2 = vam.prim(np.array([[0.8], [0.56], [0.0], [-0.028], [0.0]]), -0.05)
    assert abs(w0 + w1 + w2 - (u0 + u1) * -0.05) < 1e-15  # kinematic bed condition w_b = u_b b_x


def dyadic_hump(n, amp=0.25):
    x = (np.arange(n) + 0.5) / n
    return np.round(amp * np.exp(-((x - 0.4) ** 2) / 0.01) * 2.0**16) / 2.0**16


@pytest.mark.parametrize("bc", [(1, 1), (0, 0)])
def test_lake_at_rest_over_a_hump_bitwise(bc):
    n = 48
    b = dyadic_hump(n)
    Q = np.zeros((5, n))
    Q[0] = 1.0 - b
    R, _, p = vam.step(Q, 20, 1.0 / n, bc=bc, b=b)
    np.testing.assert_array_equal(R, Q)
    np.testing.assert_array_equal(p, 0.0)


def test_constant_bed_matches_flat():
    n, dx = 64, 1.0 / 64
    x = (np.arange(n) + 0.5) * dx
    Q = np.zeros((5, n))
    Q[0] = 1.0 + 0.1 * np.exp(-((x - 0.4) ** 2) / 0.01)
    Q[1] = Q[0] * 0.05 * np.sin(2 * np.pi * x)
    flat, tf, _ = vam.step(Q, 8, dx, bc=(1, 0))
    const, tc, _ = vam.step(Q, 8, dx, bc=(1, 0), b=np.full(n, 0.375))
    assert tc == pytest.approx(tf, rel=1e-14)
    assert np.abs(const - flat).max() < 1e-13


def test_mass_and_constraints_over_a_hump():
    n, dx = 64, 1.0 / 64
    x = (np.arange(n) + 0.5) * dx
    b = 0.3 * np.exp(-((x - 0.5) ** 2) / 0.02)
    Q = np.zeros((5, n))
    Q[0] = 1.0 + 0.05 * np.exp(-((x - 0.25) ** 2) / 0.005) - b
    Q[1] = Q[0] * 0.2
    bx = vam.bed_slope(b, dx, (1, 1))[0]
    m0 = Q[0].sum()
    for _ in range(10):
        d = 0.3 * dx / vam.wavespeed(Q, G).max()
        Qs = vam.predictor(Q, d, dx, G, (1, 1), b)
        Q, p = vam.corrector(Qs, d, dx, (1, 1), b)
        R = vam.residual(Qs, p, d, dx, (1, 1), bx)
        assert np.abs(R).max() < 1e-9 * max(1.0, np.abs(p).max())
    assert abs(Q[0].sum() - m0) / m0 < 1e-13


BED_MUTANTS = {
    "hu0_bed_force_sign": ("+ 2.0 * p1 * bx)", "- 2.0 * p1 * bx)"),
    "hu1_bed_force_dropped": (" - 6.0 * (p0 - p1) * bx)", ")"),
    "R0_bed_sign": ("2.0 * (w0 - u0 * bx)", "2.0 * (w0 + u0 * bx)"),
    "R1_bed_dropped": ("2.0 * (u1 * bx - w1)", "2.0 * (-w1)"),
    "w0_source_sign": ("Q[3] = Qs[3] + dt * 2.0 * p1", "Q[3] = Qs[3] - dt * 2.0 * p1"),
}


@pytest.mark.parametrize("name", sorted(BED_MUTANTS))
def test_bed_pins_catch_mutant(name, tmp_path):
    old, new = BED_MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "vam.py")).read()
    assert src.count(old) == 1
    path = tmp_path / f"vam_bed_{name}.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"vam_bed_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    work_ok = pressure_work_defect(mod, 400) < 1e-3
    stream_ok = slope_stream_residual(mod) < 1e-12
    assert not (work_ok and stream_ok)

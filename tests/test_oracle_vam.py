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
    "u0_pressure_sign": ("Q[1] = Qs[1] - dt * diff(h * p0, dx, bc, False)", "Q[1] = Qs[1] + dt * diff(h * p0, dx, bc, False)"),
    "w0_constraint_factor": ("u1 * dh / 3.0 + 2.0 * w0", "u1 * dh / 3.0 + w0"),
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

"""Pin P1: the oracle's basis integrals against exact rational arithmetic.

The oracle computes M, A, B, C and phi_k(0) from the Legendre three-term
recurrence and a 16-point Gauss-Legendre rule.  Here the same integrals are
taken exactly with ``fractions`` from the explicit coefficients of the shifted
Legendre polynomials, phi_k(z) = P_k(1-2z) = sum_j binom(k,j) binom(k+j,j) (-z)^j
(the basis of the "Basismatrices" class in Sec. 2.1.1 and the Legendre basis of
Sec. 3.4), so a wrong recurrence, node, index order or antiderivative fails here.
"""
from fractions import Fraction
from math import comb

import numpy as np
import pytest


def phi_coeffs(k):
    return [Fraction(comb(k, j) * comb(k + j, j) * (-1) ** j) for j in range(k + 1)]


def pmul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def pder(a):
    return [a[i] * i for i in range(1, len(a))] or [Fraction(0)]


def pint0(a):  # antiderivative vanishing at 0
    return [Fraction(0)] + [a[i] / (i + 1) for i in range(len(a))]


def integral01(a):
    return sum(c / (i + 1) for i, c in enumerate(a))


def exact_tables(N):
    m = N + 1
    phi = [phi_coeffs(k) for k in range(m)]
    dphi = [pder(p) for p in phi]
    Phi = [pint0(p) for p in phi]
    M = [integral01(pmul(phi[k], phi[k])) for k in range(m)]
    A = [[[integral01(pmul(pmul(phi[i], phi[j]), phi[k])) for k in range(m)] for j in range(m)] for i in range(m)]
    B = [[[integral01(pmul(pmul(dphi[k], phi[j]), Phi[l])) for l in range(m)] for j in range(m)] for k in range(m)]
    Cm = [[integral01(pmul(dphi[i], dphi[k])) for k in range(m)] for i in range(m)]
    p0 = [phi[k][0] for k in range(m)]
    return M, A, B, Cm, p0


@pytest.mark.parametrize("N", [0, 1, 2, 3, 4, 6])
def test_basis_tables_exact(oracle, N):
    M, A, B, Cm, p0 = oracle.basis_tables(N)
    Me, Ae, Be, Ce, p0e = exact_tables(N)
    np.testing.assert_allclose(M, [float(x) for x in Me], rtol=0, atol=1e-13)
    np.testing.assert_allclose(A, np.array(Ae, dtype=float), rtol=0, atol=1e-13)
    np.testing.assert_allclose(B, np.array(Be, dtype=float), rtol=0, atol=1e-13)
    np.testing.assert_allclose(Cm, np.array(Ce, dtype=float), rtol=0, atol=1e-11)
    np.testing.assert_allclose(p0, [float(x) for x in p0e], rtol=0, atol=0)


def test_basis_spot_values(oracle):
    M, A, B, Cm, p0 = oracle.basis_tables(4)
    np.testing.assert_allclose(M, [1, 1 / 3, 1 / 5, 1 / 7, 1 / 9], atol=1e-15)
    assert A[0, 1, 1] == pytest.approx(1 / 3, abs=1e-15)
    assert A[1, 1, 1] == pytest.approx(0.0, abs=1e-15)
    assert A[1, 1, 2] == pytest.approx(2 / 15, abs=1e-15)
    assert Cm[1, 1] == pytest.approx(4.0, abs=1e-12)
    assert Cm[2, 2] == pytest.approx(12.0, abs=1e-12)
    np.testing.assert_allclose(np.diag(Cm), [0, 4, 12, 24, 40], atol=1e-11)
    assert B[1, 1, 1] == pytest.approx(0.0, abs=1e-15)
    assert B[1, 1, 2] == pytest.approx(-1 / 15, abs=1e-15)
    assert B[1, 2, 1] == pytest.approx(1 / 15, abs=1e-15)
    np.testing.assert_array_equal(p0, np.ones(5))


def test_basis_selection_rules(oracle):
    """A_ijk vanishes unless i+j+k is even and |i-j| <= k <= i+j; B_k0l = -delta_kl M_k (k,l >= 1)."""
    N = 5
    M, A, B, Cm, p0 = oracle.basis_tables(N)
    for i in range(N + 1):
        for j in range(N + 1):
            for k in range(N + 1):
                allowed = (i + j + k) % 2 == 0 and abs(i - j) <= k <= i + j
                if not allowed:
                    assert abs(A[i, j, k]) < 1e-14
                else:
                    assert abs(A[i, j, k]) > 1e-6
    for k in range(1, N + 1):
        for l in range(1, N + 1):
            assert B[k, 0, l] == pytest.approx(-M[k] if k == l else 0.0, abs=1e-14)
    # phi_0' = 0: no bulk coupling of the mean
    assert np.all(np.abs(B[0]) < 1e-15) and np.all(np.abs(Cm[0]) < 1e-15)

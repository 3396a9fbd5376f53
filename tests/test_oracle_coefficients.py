"""Pins of the oracle's 1-D Riesz stiffness coefficients (Sec. 2) against independent facts."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import p1, sfde


def _riesz_bilinear_quadrature(n, rho, i, j, length=1.0):
    """K/(2cos) [(D_L phi_j, D_R phi_i) + (D_R phi_j, D_L phi_i)] with K = 1, by adaptive quadrature.

    The one-sided Riemann-Liouville derivatives of the ramps (x-c)_+ and (c-x)_+ follow from the
    power rule, D^rho (x-c)^1 = (x-c)^{1-rho} / Gamma(2-rho); a hat is a second difference of ramps.
    """
    h = length / (n + 1)
    x = h * np.arange(n + 2)
    gm = math.gamma(2.0 - rho)

    def dl(k, s):  # left derivative of hat k (interior index k -> node k+1)
        c = x[k + 1]
        f = lambda v: max(v, 0.0) ** (1.0 - rho)
        return (f(s - c + h) - 2.0 * f(s - c) + f(s - c - h)) / (h * gm)

    def dr(k, s):
        c = x[k + 1]
        f = lambda v: max(v, 0.0) ** (1.0 - rho)
        return (f(c + h - s) - 2.0 * f(c - s) + f(c - h - s)) / (h * gm)

    pts = list(x)
    t1 = quad(lambda s: dl(j, s) * dr(i, s), 0.0, length, points=pts, limit=400, epsabs=1e-14, epsrel=1e-12)[0]
    t2 = quad(lambda s: dr(j, s) * dl(i, s), 0.0, length, points=pts, limit=400, epsabs=1e-14, epsrel=1e-12)[0]
    return (t1 + t2) / (2.0 * math.cos(rho * math.pi))


@pytest.mark.parametrize("rho", [0.55, 0.7, 0.95])
def test_coefficients_match_quadrature_of_bilinear_form(rho):
    n = 6
    a = sfde.riesz_coefficients(n, rho)
    for j in range(n):
        q = _riesz_bilinear_quadrature(n, rho, 0, j)
        assert abs(q - a[j]) <= 1e-8 * abs(a[0]), (j, q, a[j])


@pytest.mark.parametrize("rho", [0.6, 0.75, 0.95])
def test_paper_printed_blocks_collapse_to_1d_coefficients(rho):
    """A_1 + A_2 + A_2^T (the paper's printed entries, Sec. 2) = (4-2rho)(g(l)+g(-l))."""
    n = 14
    h = 1.0 / (n + 1)
    a = sfde.riesz_coefficients(n, rho)
    pref = h ** (1 - 2 * rho) / (2 * math.cos(rho * math.pi) * math.gamma(4 - 2 * rho))
    for l in range(n):
        lhs = p1.a1(l, rho) + p1.a2_upper(l, rho) + (p1.a2_lower(l, rho) if l else p1.a2_upper(0, rho))
        rhs = (4 - 2 * rho) * a[l] / pref
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs)), (l, lhs, rhs)


def test_rho_one_is_textbook_laplacian():
    n = 9
    h = 1.0 / (n + 1)
    A = sfde.stiffness_1d(n, 1.0)
    ref = (2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)) / h
    np.testing.assert_allclose(A, ref, rtol=0, atol=1e-12 / h)


@pytest.mark.parametrize("rho", [0.55, 0.8])
def test_large_k_asymptotics(rho):
    """For k >= 2, g(k) is the 4th central difference of k^p (p = 3-2rho):
    g(k) = p(p-1)(p-2)(p-3) k^{p-4} [1 + (p-4)(p-5)/(6 k^2) + O(k^-4)]."""
    n = 1024
    h = 1.0 / (n + 1)
    a = sfde.riesz_coefficients(n, rho)
    p = 3 - 2 * rho
    pref = h ** (1 - 2 * rho) / (2 * math.cos(rho * math.pi) * math.gamma(4 - 2 * rho))
    for k in (300, 700, 1023):
        lead = pref * p * (p - 1) * (p - 2) * (p - 3) * k ** (p - 4)
        corr = 1 + (p - 4) * (p - 5) / (6 * k * k)
        assert abs(a[k] / lead - corr) < 2e-9, (k, a[k] / lead, corr)


@pytest.mark.parametrize("rho", [0.51, 0.6, 0.9, 0.99])
def test_symmetric_toeplitz_positive_definite(rho):
    n = 40
    A = sfde.stiffness_1d(n, rho)
    assert np.array_equal(A, A.T)
    assert np.all(A[1:, 1:] == A[:-1, :-1])
    np.linalg.cholesky(A)
    assert np.linalg.eigvalsh(A).min() > 0
    a = sfde.riesz_coefficients(n, rho)
    assert a[0] > 0 and np.all(a[1:] < 0)  # off-diagonal entries of a Riesz stiffness are negative


def test_mpmath_definition():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for rho in (0.6, 0.95):
        n = 200
        a = sfde.riesz_coefficients(n, rho)
        h = mp.mpf(1) / (n + 1)
        r = mp.mpf(repr(rho))
        p = 3 - 2 * r
        c = (1, -4, 6, -4, 1)
        pw = lambda v: mp.mpf(0) if v <= 0 else mp.mpf(v) ** p
        pref = h ** (1 - 2 * r) / (2 * mp.cos(r * mp.pi) * mp.gamma(4 - 2 * r))
        for k in (0, 1, 2, 5, 77, 199):
            g = sum(cc * (pw(k + s) + pw(-k + s)) for s, cc in zip(range(-2, 3), c))
            assert abs(float(pref * g) - a[k]) <= 2e-15 * abs(a[k])

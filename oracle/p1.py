"""The paper's P1-triangle Toeplitz blocks A_1^rho, A_2^rho (Sec. 2) -- FP64 CPU oracle.

Test infrastructure only.  The 2-D stiffness of Sec. 2 is
A_x^beta = h_x^{1-2beta} h_y / (2 cos(beta pi) Gamma(5-2beta)) [I (x) A_1 + E (x) A_2 + E^T (x) A_2^T]
with Toeplitz blocks whose entries are printed in closed form.  Integrating a P1 hat over y
collapses the block row to A_1 + A_2 + A_2^T, which must equal (4-2 rho) times the 1-D
linear-element entries g(k)+g(-k) used by ``oracle.sfde`` -- the link between the paper's
printed formulas and the tensor-product operator of this project (tested).

Entries are evaluated here exactly as printed, in 40-digit decimal arithmetic.
"""
from __future__ import annotations

from decimal import Decimal, getcontext


def _pw(v, e):
    v = Decimal(v)
    return Decimal(0) if v <= 0 else v ** e


def a1(l: int, rho: float) -> float:
    """Entry a^{1,rho}_{k,k+l} = a^{1,rho}_{k+l,k} of A_1^rho (symmetric Toeplitz), l >= 0."""
    getcontext().prec = 40
    r = Decimal(repr(float(rho)))
    p3, p4 = 3 - 2 * r, 4 - 2 * r
    if l == 0:
        return float(Decimal(2) ** (6 - 2 * r) + 16 * r - 40)
    if l == 1:
        return float(2 * Decimal(3) ** (4 - 2 * r) + (2 * r - 6) * Decimal(2) ** (5 - 2 * r) - 16 * r + 34)
    v = (4 * (4 - 2 * r) * (-_pw(l - 1, p3) + 2 * _pw(l, p3) - _pw(l + 1, p3))
         - 2 * _pw(l - 2, p4) + 4 * _pw(l - 1, p4) - 4 * _pw(l + 1, p4) + 2 * _pw(l + 2, p4))
    return float(v)


def a2_upper(l: int, rho: float) -> float:
    """Entry a^{2,rho}_{k,k+l} of A_2^rho on or above the diagonal, l >= 0."""
    getcontext().prec = 40
    r = Decimal(repr(float(rho)))
    p3, p4 = 3 - 2 * r, 4 - 2 * r
    if l in (0, 1):
        return float(4 - Decimal(2) ** (4 - 2 * r) * r)
    v = ((4 - 2 * r) * (_pw(l - 2, p3) - _pw(l - 1, p3) - _pw(l, p3) + _pw(l + 1, p3))
         + 2 * _pw(l - 2, p4) - 6 * _pw(l - 1, p4) + 6 * _pw(l, p4) - 2 * _pw(l + 1, p4))
    return float(v)


def a2_lower(m: int, rho: float) -> float:
    """Entry a^{2,rho}_{p+m,p} of A_2^rho below the diagonal, m >= 1."""
    getcontext().prec = 40
    r = Decimal(repr(float(rho)))
    p3, p4 = 3 - 2 * r, 4 - 2 * r
    v = ((4 - 2 * r) * (_pw(m - 1, p3) - _pw(m, p3) - _pw(m + 1, p3) + _pw(m + 2, p3))
         + 2 * _pw(m - 1, p4) - 6 * _pw(m, p4) + 6 * _pw(m + 1, p4) - 2 * _pw(m + 2, p4))
    return float(v)

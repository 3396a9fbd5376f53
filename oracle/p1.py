"""The paper's P1-triangle operator (Sec. 2) -- FP64 CPU oracle.

Test infrastructure only.  Contents:
* the printed Toeplitz entries of A_1^rho, A_2^rho, evaluated as printed in 40-digit decimal
  arithmetic.  The 2-D stiffness is
  A_x^beta = h_x^{1-2beta} h_y / (2 cos(beta pi) Gamma(5-2beta)) [I (x) A_1 + E (x) A_2 + E^T (x) A_2^T];
  integrating a P1 hat over y collapses the block row to A_1 + A_2 + A_2^T, which must equal
  (4-2 rho) times the 1-D linear-element entries g(k)+g(-k) used by ``oracle.sfde`` -- the link
  between the printed formulas and the tensor-product operator (tested);
* the assembled matrices M_h, A_x^beta, A_y^gamma exactly as printed (A_y through the printed
  permutation list pi), the fully discrete scheme (2.4) with them and its sequential stepping by
  dense Cholesky solves (small N only);
* the L2 error of the P1 interpolant (the error norm of Tables 1-4).
"""
from __future__ import annotations

import math
from decimal import Decimal, getcontext

import numpy as np


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


# ---------------------------------------------------------------------------- assembled operators
#
# Unknowns are the interior nodes of the uniform triangulation of Sec. 2, numbered x fastest:
# index(i, j) = j * N_x + i, U[j, i] = u(x_i, y_j).  The triangles cut every cell along its
# south-west to north-east diagonal: this is the mesh whose mass matrix is the printed
# block-tridiagonal M_h (its off-diagonal block M_2 couples node (i, j) with (i, j+1) and (i+1, j+1)).


def toeplitz_blocks(n: int, rho: float):
    """Dense (n x n) A_1^rho (symmetric Toeplitz) and A_2^rho (Toeplitz, not symmetric) from the
    printed entries (Sec. 2)."""
    a1v = [a1(l, rho) for l in range(n)]
    up = [a2_upper(l, rho) for l in range(n)]
    lo = [0.0] + [a2_lower(m, rho) for m in range(1, n)]
    A1 = np.empty((n, n))
    A2 = np.empty((n, n))
    for i in range(n):
        for j in range(n):
            A1[i, j] = a1v[abs(i - j)]
            A2[i, j] = up[j - i] if j >= i else lo[i - j]
    return A1, A2


def _block_tridiag(nb: int, D, U):
    """Block tridiagonal matrix with nb diagonal blocks D, super-diagonal blocks U and sub-diagonal
    blocks U^T."""
    E = np.eye(nb, k=1)
    return np.kron(np.eye(nb), D) + np.kron(E, U) + np.kron(E.T, U.T)


def mass_p1(nx: int, ny: int, hx: float, hy: float):
    """M_h = (h_x h_y / 12) blocktridiag(M_2^T, M_1, M_2), M_1 = tridiag(1, 6, 1), M_2 upper
    bidiagonal with ones (Sec. 2); (N_x N_y) square."""
    M1 = 6.0 * np.eye(nx) + np.eye(nx, k=1) + np.eye(nx, k=-1)
    M2 = np.eye(nx) + np.eye(nx, k=1)
    return (hx * hy / 12.0) * _block_tridiag(ny, M1, M2)


def stiffness_p1_x(beta: float, nx: int, ny: int, hx: float, hy: float):
    """A_x^beta = h_x^{1-2 beta} h_y / (2 cos(beta pi) Gamma(5 - 2 beta)) blocktridiag((A_2)^T, A_1, A_2)
    with (N_y) blocks of order N_x (Sec. 2)."""
    A1, A2 = toeplitz_blocks(nx, beta)
    c = hx ** (1.0 - 2.0 * beta) * hy / (2.0 * math.cos(beta * math.pi) * math.gamma(5.0 - 2.0 * beta))
    return c * _block_tridiag(ny, A1, A2)


def permutation_pi(nx: int, ny: int) -> np.ndarray:
    """The index list pi of Sec. 2 (0-based): for x index i = 1..N_x the y-line of nodes
    i, i + N_x, ..., i + (N_y - 1) N_x, i.e. the unknowns renumbered y fastest."""
    return np.array([i + j * nx for i in range(nx) for j in range(ny)], dtype=np.int64)


def stiffness_p1_y(gamma: float, nx: int, ny: int, hx: float, hy: float):
    """A_y^gamma = h_x h_y^{1-2 gamma} / (2 cos(gamma pi) Gamma(5 - 2 gamma)) P_pi^T blocktridiag(...) P_pi
    with (N_x) blocks of order N_y (Sec. 2), P_pi the permutation matrix of the list pi
    ((P_pi u)_k = u_{pi(k)})."""
    A1, A2 = toeplitz_blocks(ny, gamma)
    c = hx * hy ** (1.0 - 2.0 * gamma) / (2.0 * math.cos(gamma * math.pi) * math.gamma(5.0 - 2.0 * gamma))
    B = _block_tridiag(nx, A1, A2)
    n = nx * ny
    P = np.zeros((n, n))
    P[np.arange(n), permutation_pi(nx, ny)] = 1.0
    return c * (P.T @ B @ P)


class P1SFDE:
    """The fully discrete scheme (2.4) with the paper's P1-triangle matrices M_h, A_x^beta, A_y^gamma,
    assembled densely (small N only).  Fields U are (N_y, N_x) arrays."""

    def __init__(self, beta, gamma, kx, ky, nx, ny, t, omega=(0.0, 1.0, 0.0, 1.0)):
        a, b, c, d = omega
        self.beta, self.gamma, self.kx, self.ky = float(beta), float(gamma), float(kx), float(ky)
        self.nx, self.ny = int(nx), int(ny)
        self.t = np.asarray(t, dtype=np.float64)
        self.nt = len(self.t) - 1
        self.hx, self.hy = (b - a) / (nx + 1), (d - c) / (ny + 1)
        self.M = mass_p1(nx, ny, self.hx, self.hy)
        self.K = (self.kx * stiffness_p1_x(beta, nx, ny, self.hx, self.hy)
                  + self.ky * stiffness_p1_y(gamma, nx, ny, self.hx, self.hy))
        self._chol = {}

    def apply_S(self, U, tau):
        return ((self.M + tau * self.K) @ U.reshape(-1)).reshape(self.ny, self.nx)

    def apply_B(self, U, tau):
        return ((self.M - tau * self.K) @ U.reshape(-1)).reshape(self.ny, self.nx)

    def solve_S(self, R, tau):
        """S X = R, S = M_h + tau K (symmetric positive definite, Lemma 3.2), by Cholesky."""
        from scipy.linalg import cho_factor, cho_solve
        key = float(tau)
        if key not in self._chol:
            self._chol[key] = cho_factor(self.M + tau * self.K)
        return cho_solve(self._chol[key], R.reshape(-1)).reshape(self.ny, self.nx)

    def step(self, U, n, F=None, dense=True):
        """Phi_n(U) = S_n^{-1}(B_n U + F_n), tau_n = (t_n - t_{n-1}) / 2 (Eq. (2.4)).  (``dense`` is
        accepted for the interface of ``oracle.mgrit``; the solve is always the dense one.)"""
        tau = 0.5 * (self.t[n] - self.t[n - 1])
        R = self.apply_B(U, tau)
        if F is not None:
            R = R + F
        return self.solve_S(R, tau)

    def propagate(self, U, dt, scheme="cn", dense=True):
        """Homogeneous one-step propagators: CN (M_h + dt/2 K)^{-1}(M_h - dt/2 K) (Eq. (3.4)) or
        backward Euler (M_h + dt K)^{-1} M_h."""
        if scheme == "cn":
            return self.solve_S(self.apply_B(U, 0.5 * dt), 0.5 * dt)
        if scheme == "be":
            return self.solve_S((self.M @ U.reshape(-1)).reshape(self.ny, self.nx), dt)
        raise ValueError(scheme)


def seq_timestep_p1(prob: P1SFDE, U0, forcing=None, keep_all=True):
    """Sequential time stepping U_n = Phi_n(U_{n-1}), n = 1..N_t, with the P1 operator; ``forcing``
    is any object whose dense(n) returns F_n (or None)."""
    U = np.asarray(U0, dtype=np.float64).copy()
    out = [U.copy()] if keep_all else None
    for n in range(1, prob.nt + 1):
        U = prob.step(U, n, None if forcing is None else forcing.dense(n))
        if keep_all:
            out.append(U.copy())
    return np.stack(out) if keep_all else U


# ---------------------------------------------------------------------------- error norm

def _duffy_rule(k: int):
    """Points (s, r) and weights of a collapsed Gauss-Legendre rule on the reference triangle
    {s >= 0, r >= 0, s + r <= 1} (k x k points, exact for polynomials of degree <= 2k - 2)."""
    g, w = np.polynomial.legendre.leggauss(k)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    s = np.repeat(g, k)
    v = np.tile(g, k)
    ws = np.repeat(w, k) * np.tile(w, k)
    # (s, v) in the unit square -> (s, (1 - s) v) in the triangle, Jacobian (1 - s)
    return s, (1.0 - s) * v, ws * (1.0 - s)


def l2_error_p1(U, exact, omega=(0.0, 1.0, 0.0, 1.0), k: int = 10):
    """|| u - I_h U ||_{L^2(Omega)} with I_h the P1 interpolant of the nodal values on the
    triangulation above (zero on the boundary); a collapsed 10 x 10 Gauss rule per triangle."""
    a, b, c, d = omega
    ny, nx = U.shape
    hx, hy = (b - a) / (nx + 1), (d - c) / (ny + 1)
    Z = np.zeros((ny + 2, nx + 2))
    Z[1:-1, 1:-1] = U
    s, r, w = _duffy_rule(k)
    x0 = a + hx * np.arange(nx + 1)
    y0 = c + hy * np.arange(ny + 1)
    X0, Y0 = np.meshgrid(x0, y0)       # lower-left corner of every cell, (ny+1, nx+1)
    u00, u10 = Z[:-1, :-1], Z[:-1, 1:]
    u01, u11 = Z[1:, :-1], Z[1:, 1:]
    tot = 0.0
    for sq, rq, wq in zip(s, r, w):
        # lower-right triangle (0,0), (1,0), (1,1): local point (s + r, r)
        xl, yl = sq + rq, rq
        v = u00 + (u10 - u00) * xl + (u11 - u10) * yl
        e = exact(X0 + xl * hx, Y0 + yl * hy) - v
        tot += wq * float((e * e).sum())
        # upper-left triangle (0,0), (1,1), (0,1): local point (r, s + r)
        xl, yl = rq, sq + rq
        v = u00 + (u11 - u01) * xl + (u01 - u00) * yl
        e = exact(X0 + xl * hx, Y0 + yl * hy) - v
        tot += wq * float((e * e).sum())
    return math.sqrt(tot * hx * hy)

"""Spatial operators and sequential time stepping (FP64 CPU oracle; test infrastructure only).

Discretisation followed (paper Sec. 2):

* Riesz derivative d^{2rho}u/d|x|^{2rho} = -(D_L^{2rho} + D_R^{2rho}) u / (2 cos(rho pi))  (Sec. 1).
* Weak form (Eq. (2.2)): the stiffness bilinear form of one direction is
  K/(2 cos(rho pi)) [(D_L^rho u, D_R^rho v) + (D_R^rho u, D_L^rho v)].
* Linear hat functions on a uniform grid.  For hats, the left derivative of the ramp
  (x-c)_+ is (x-c)_+^{1-rho}/Gamma(2-rho) and the right one of (c-x)_+ is
  (c-x)_+^{1-rho}/Gamma(2-rho); their product integrates to a Beta function, so
  (D_L^rho phi_j, D_R^rho phi_i) = h^{1-2rho}/Gamma(4-2rho) * g(i-j) with
  g(k) = sum_{s=-2..2} c_s (k+s)_+^{3-2rho}, c = (1,-4,6,-4,1).
  Hence the 1-D stiffness is the symmetric Toeplitz matrix
  A[i,j] = a_{|i-j|},  a_k = h^{1-2rho} (g(k)+g(-k)) / (2 cos(rho pi) Gamma(4-2rho)).
  This is the 1-D reduction of the paper's closed forms for A_1, A_2 (checked in the tests
  against those printed formulas and against brute-force quadrature).
* 1-D mass matrix M = (h/6) tridiag(1,4,1).
* Tensor-product (bilinear) elements in 2-D: for U[j,i] = u(x_i, y_j),
      M_h U       = M_y U M_x,
      K U         = K_x M_y U A_x + K_y A_y U M_x,
  and the fully discrete step of Eq. (2.4) with tau_n = (t_n - t_{n-1})/2:
      S_n U_n = B_n U_{n-1} + F_n,   S_n = M_h + tau_n K,  B_n = M_h - tau_n K.

Parity pins (tests/test_oracle_*.py): coefficients against 40-digit arithmetic of the
definition, against numerical quadrature of the bilinear form, against the paper's printed
A_1/A_2 entries, the rho -> 1 limit (textbook Laplacian); the FDM step against a dense
Kronecker solve; the modal recurrence against stepping; the O(h^2 + tau^2) saturation order
on the manufactured solution of Example 4.1.
"""
from __future__ import annotations

import math
from decimal import Decimal, getcontext
from functools import lru_cache

import numpy as np
import scipy.linalg as sla

_C5 = (1, -4, 6, -4, 1)


@lru_cache(maxsize=64)
def _g_sym_decimal(n: int, rho: float) -> tuple:
    """g(k) + g(-k), k = 0..n-1, evaluated in 40-digit decimal arithmetic.

    g(k) = sum_{s=-2}^{2} c_s (k+s)_+^{3-2rho}: a fourth difference of |k|^{3-2rho}, which
    cancels badly in binary FP64 for large k, so the oracle evaluates the definition with
    40 significant digits and rounds once.
    """
    getcontext().prec = 40
    p = Decimal(3) - 2 * Decimal(repr(float(rho)))

    def pw(v: int) -> Decimal:
        return Decimal(0) if v <= 0 else Decimal(v) ** p

    out = []
    for k in range(n):
        s = Decimal(0)
        for off, c in zip(range(-2, 3), _C5):
            s += c * (pw(k + off) + pw(-k + off))
        out.append(float(s))
    return tuple(out)


def riesz_coefficients(n: int, rho: float, length: float = 1.0) -> np.ndarray:
    """a_k, k = 0..n-1, of the 1-D linear-element Riesz stiffness (Sec. 2, Eq. (2.2))."""
    if not (0.5 < rho <= 1.0):
        raise ValueError("rho must lie in (1/2, 1]")
    h = length / (n + 1)
    pref = h ** (1.0 - 2.0 * rho) / (2.0 * math.cos(rho * math.pi) * math.gamma(4.0 - 2.0 * rho))
    return pref * np.array(_g_sym_decimal(n, float(rho)), dtype=np.float64)


def stiffness_1d(n: int, rho: float, length: float = 1.0) -> np.ndarray:
    """Dense symmetric Toeplitz A with A[i,j] = a_{|i-j|}."""
    return sla.toeplitz(riesz_coefficients(n, rho, length))


def mass_1d(n: int, length: float = 1.0) -> np.ndarray:
    """1-D linear-element mass matrix (h/6) tridiag(1,4,1)."""
    h = length / (n + 1)
    return (h / 6.0) * (4.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1))


class SFDE:
    """One instance of the fully discrete problem (Eq. (2.4)) with Kronecker operators.

    Fields U are (N_y, N_x) arrays, U[j,i] = u(x_i, y_j).
    """

    def __init__(self, beta, gamma, kx, ky, nx, ny, t, omega=(0.0, 1.0, 0.0, 1.0)):
        a, b, c, d = omega
        self.beta, self.gamma, self.kx, self.ky = float(beta), float(gamma), float(kx), float(ky)
        self.nx, self.ny = int(nx), int(ny)
        self.t = np.asarray(t, dtype=np.float64)
        self.nt = len(self.t) - 1
        self.omega = tuple(omega)
        self.Ax = stiffness_1d(nx, beta, b - a)
        self.Ay = stiffness_1d(ny, gamma, d - c)
        self.Mx = mass_1d(nx, b - a)
        self.My = mass_1d(ny, d - c)
        self._eig = None

    # ---- operators (Sec. 2)
    def apply_mass(self, U):
        return self.My @ U @ self.Mx

    def apply_stiff(self, U):
        return self.kx * (self.My @ U @ self.Ax) + self.ky * (self.Ay @ U @ self.Mx)

    def apply_S(self, U, tau):
        return self.apply_mass(U) + tau * self.apply_stiff(U)

    def apply_B(self, U, tau):
        return self.apply_mass(U) - tau * self.apply_stiff(U)

    def kron_S(self, tau):
        """Assembled S = M_y(x)M_x + tau (K_x M_y(x)A_x + K_y A_y(x)M_x), row-major vec."""
        return (np.kron(self.My, self.Mx)
                + tau * (self.kx * np.kron(self.My, self.Ax) + self.ky * np.kron(self.Ay, self.Mx)))

    # ---- generalised eigenpairs A V = M V diag(lam), V^T M V = I
    def eig(self):
        if self._eig is None:
            lx, Vx = sla.eigh(self.Ax, self.Mx)
            ly, Vy = sla.eigh(self.Ay, self.My)
            self._eig = (lx, Vx, ly, Vy)
        return self._eig

    def sigma(self):
        """sigma[j,i] = K_x lam_x[i] + K_y lam_y[j]: eigenvalues of M_h^{-1} K (Eq. (3.5))."""
        lx, _, ly, _ = self.eig()
        return self.kx * lx[None, :] + self.ky * ly[:, None]

    # ---- one step solve
    def solve_S_dense(self, R, tau):
        """S X = R by a dense solve of the assembled Kronecker matrix (tiny sizes only)."""
        x = np.linalg.solve(self.kron_S(tau), R.reshape(-1))
        return x.reshape(self.ny, self.nx)

    def solve_S_fdm(self, R, tau):
        """S X = R by fast diagonalisation: X = V_y [(V_y^T R V_x) / (1 + tau sigma)] V_x^T."""
        _, Vx, _, Vy = self.eig()
        return Vy @ ((Vy.T @ R @ Vx) / (1.0 + tau * self.sigma())) @ Vx.T

    def step(self, U, n, F=None, dense=False):
        """Phi_n(U) = S_n^{-1}(B_n U + F_n), the fine step of Eq. (2.4), n = 1..N_t."""
        tau = 0.5 * (self.t[n] - self.t[n - 1])
        R = self.apply_B(U, tau)
        if F is not None:
            R = R + F
        return self.solve_S_dense(R, tau) if dense else self.solve_S_fdm(R, tau)

    def propagate(self, U, dt, scheme="cn", dense=False):
        """Homogeneous one-step propagator with step dt.

        scheme "cn": Psi = (M_h + dt/2 K)^{-1}(M_h - dt/2 K), Eqs. (3.2) and (3.4);
        scheme "be": Psi = (M_h + dt K)^{-1} M_h (L-stable rediscretisation).
        """
        if scheme == "cn":
            tau = 0.5 * dt
            R = self.apply_B(U, tau)
        elif scheme == "be":
            tau = dt
            R = self.apply_mass(U)
        else:
            raise ValueError(scheme)
        return self.solve_S_dense(R, tau) if dense else self.solve_S_fdm(R, tau)


def dense_forcing(forcing, n):
    return None if forcing is None else forcing.dense(n)


def seq_timestep(prob: SFDE, U0, forcing=None, dense=False, keep_all=True):
    """Sequential time stepping U_n = Phi_n(U_{n-1}), n = 1..N_t (Eq. (2.4)).

    Returns an (N_t+1, N_y, N_x) array (or only U_{N_t} if keep_all is False).
    """
    U = np.asarray(U0, dtype=np.float64).copy()
    out = [U.copy()] if keep_all else None
    for n in range(1, prob.nt + 1):
        U = prob.step(U, n, dense_forcing(forcing, n), dense=dense)
        if keep_all:
            out.append(U.copy())
    return np.stack(out) if keep_all else U


def modal_lambda(sigma, dt, scheme="cn"):
    """Eigenvalues of the one-step propagator: (2 - dt s)/(2 + dt s) for CN (Eq. (3.7)),
    1/(1 + dt s) for backward Euler."""
    if scheme == "cn":
        return (2.0 - dt * sigma) / (2.0 + dt * sigma)
    if scheme == "be":
        return 1.0 / (1.0 + dt * sigma)
    raise ValueError(scheme)


def spectral_sequential_iter(prob: SFDE, U0, forcing=None, keep=None):
    """Exact sequential solution through the per-mode recurrence of Eq. (3.7), one time point at a
    time: yields (n, U_n) for n = 0..N_t (only the n in ``keep`` when it is given; the recurrence still
    runs over every step).

    With C_n = V_y^T M_y U_n M_x V_x (so U_n = V_y C_n V_x^T), each mode obeys
    c_n = lambda_n c_{n-1} + f_n / (1 + tau_n sigma), f_n = (V_y^T F_n V_x).  ``forcing`` is separable
    (factors time_w, bx, by) or any object whose dense(n) returns F_n.
    """
    lx, Vx, ly, Vy = prob.eig()
    sig = prob.sigma()
    Wx, Wy = prob.Mx @ Vx, prob.My @ Vy
    U0 = np.asarray(U0, dtype=np.float64)
    C = Wy.T @ U0 @ Wx
    keep = None if keep is None else set(keep)
    if keep is None or 0 in keep:
        yield 0, U0.copy()
    separable = forcing is not None and hasattr(forcing, "bx")
    if separable:
        px = forcing.bx @ Vx  # (R, N_x): V_x^T b_x^r
        py = forcing.by @ Vy  # (R, N_y)
    for n in range(1, prob.nt + 1):
        dt = prob.t[n] - prob.t[n - 1]
        C = modal_lambda(sig, dt) * C
        if forcing is not None:
            if separable:
                fh = np.einsum("r,rj,ri->ji", forcing.time_w[n - 1], py, px)
            else:
                fh = Vy.T @ forcing.dense(n) @ Vx
            C = C + fh / (1.0 + 0.5 * dt * sig)
        if keep is None or n in keep:
            yield n, Vy @ C @ Vx.T


def spectral_sequential(prob: SFDE, U0, forcing=None, keep=None):
    """``spectral_sequential_iter`` collected: a dict n -> U_n for the time indices in ``keep``
    (default: all)."""
    return dict(spectral_sequential_iter(prob, U0, forcing, keep))


# ---------------------------------------------------------------------------- error norms

_GQ_X, _GQ_W = np.polynomial.legendre.leggauss(6)


def l2_error_bilinear(U, exact, omega=(0.0, 1.0, 0.0, 1.0)):
    """|| u - I_h U ||_{L^2(Omega)} with I_h the bilinear interpolant of the nodal values
    (zero on the boundary), by a 6x6 Gauss rule per element."""
    a, b, c, d = omega
    ny, nx = U.shape
    hx, hy = (b - a) / (nx + 1), (d - c) / (ny + 1)
    Z = np.zeros((ny + 2, nx + 2))
    Z[1:-1, 1:-1] = U
    s = 0.5 * (1.0 + _GQ_X)
    w = 0.5 * _GQ_W
    tot = 0.0
    xs = a + hx * np.arange(nx + 1)
    ys = c + hy * np.arange(ny + 1)
    for qy, wy in zip(s, w):
        for qx, wx in zip(s, w):
            X = xs[None, :] + qx * hx
            Y = ys[:, None] + qy * hy
            uh = ((1 - qx) * (1 - qy) * Z[:-1, :-1] + qx * (1 - qy) * Z[:-1, 1:]
                  + (1 - qx) * qy * Z[1:, :-1] + qx * qy * Z[1:, 1:])
            tot += wx * wy * np.sum((exact(X, Y) - uh) ** 2)
    return math.sqrt(tot * hx * hy)

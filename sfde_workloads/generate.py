"""Seeded problem data for the 2-D Riesz SFDE (no solver arithmetic here).

Layout conventions shared by every consumer:

* interior nodes x_i = a + i*h_x, i = 1..N_x, h_x = (b-a)/(N_x+1); same in y;
* a spatial field is an array of shape (N_y, N_x): ``U[j, i] = u(x_i, y_j)``;
* a time grid is ``t[0..N_t]`` with t[0] = 0, strictly increasing;
* a separable load ``Forcing(time_w, bx, by)`` means
  ``F_n[j, i] = sum_r time_w[n-1, r] * by[r, j] * bx[r, i]`` for n = 1..N_t,
  i.e. the space-time integral defined below Eq. (2.4) for a source f = sum_r c_r(t) f^r_x(x) f^r_y(y),
  with time_w[n-1, r] = int_{I_n} c_r dt, bx[r, i] = (f^r_x, phi_i), by[r, j] = (f^r_y, phi_j).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np


# ----------------------------------------------------------------------------- grids

def interior_nodes(n: int, lo: float, hi: float) -> np.ndarray:
    """Interior nodes of a uniform partition of (lo, hi) into n+1 intervals (Sec. 2)."""
    h = (hi - lo) / (n + 1)
    return lo + h * np.arange(1, n + 1, dtype=np.float64)


def time_grid(nt: int, T: float = 1.0, kind: str = "uniform", eps: float | None = None) -> np.ndarray:
    """Temporal partition 0 = t_0 < ... < t_N = T (Sec. 2, Sec. 4.1).

    kind = "uniform"  : t_n = T n / N;
           "graded"   : t_n = T (n/N)^2, so the fine propagator depends on n;
           "shishkin" : the piecewise-uniform partition of Sec. 4.1 with N/4 steps on
                        [0, s], N/2 on [s, T-s] and N/4 on [T-s, T], s = 2 eps ln N (scaled by T).
    """
    if nt < 1:
        raise ValueError("nt must be >= 1")
    n = np.arange(nt + 1, dtype=np.float64)
    if kind == "uniform":
        t = T * n / nt
    elif kind == "graded":
        t = T * (n / nt) ** 2
    elif kind == "shishkin":
        if nt % 4 or eps is None:
            raise ValueError("shishkin grid needs nt % 4 == 0 and eps")
        s = min(2.0 * eps * math.log(nt), 0.25) * T
        q = nt // 4
        t = np.concatenate([
            np.linspace(0.0, s, q + 1)[:-1],
            np.linspace(s, T - s, 2 * q + 1)[:-1],
            np.linspace(T - s, T, q + 1),
        ])
    else:
        raise ValueError(f"unknown time grid kind {kind!r}")
    t[0] = 0.0
    t[-1] = T
    return t


# ----------------------------------------------------------------------------- initial data

def sine_mode_amplitudes(seed: int, pmax: int = 4) -> np.ndarray:
    """Amplitudes a[p-1, q-1] = N(0,1)/(p^2+q^2), p,q = 1..pmax, drawn with PCG64(seed)."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((pmax, pmax))
    p = np.arange(1, pmax + 1, dtype=np.float64)
    return z / (p[:, None] ** 2 + p[None, :] ** 2)


def sine_mode_nodal(amp: np.ndarray, nx: int, ny: int, omega=(0.0, 1.0, 0.0, 1.0)) -> np.ndarray:
    """psi_0(x,y) = sum_{p,q} a_pq sin(p pi x') sin(q pi y') sampled at interior nodes, (N_y, N_x)."""
    a, b, c, d = omega
    x = (interior_nodes(nx, a, b) - a) / (b - a)
    y = (interior_nodes(ny, c, d) - c) / (d - c)
    P = amp.shape[0]
    sx = np.sin(np.pi * np.outer(np.arange(1, P + 1), x))  # (P, nx)
    sy = np.sin(np.pi * np.outer(np.arange(1, amp.shape[1] + 1), y))  # (Q, ny)
    return sy.T @ amp.T @ sx  # sum_pq a_pq sy[q, j] sx[p, i]


# ----------------------------------------------------------------------------- loads

@dataclass
class Forcing:
    """Separable load: F_n[j,i] = sum_r time_w[n-1,r] by[r,j] bx[r,i], n = 1..N_t."""
    time_w: np.ndarray  # (N_t, R)
    bx: np.ndarray      # (R, N_x)
    by: np.ndarray      # (R, N_y)

    @property
    def rank(self) -> int:
        return self.bx.shape[0]

    def dense(self, n: int) -> np.ndarray:
        """F_n as an (N_y, N_x) array (n = 1..N_t)."""
        return np.einsum("r,rj,ri->ji", self.time_w[n - 1], self.by, self.bx)


def _load_second_difference(antider, nodes: np.ndarray, h: float) -> np.ndarray:
    """(f, phi_i) for a hat phi_i of width 2h from an antiderivative G with G'' = f.

    Two integrations by parts give (f, phi_i) = (G(x_{i-1}) - 2 G(x_i) + G(x_{i+1})) / h.
    """
    return (antider(nodes - h) - 2.0 * antider(nodes) + antider(nodes + h)) / h


def _w_antider(z):
    # w(z) = z^2 (1-z)^2 = z^2 - 2 z^3 + z^4 ; G'' = w
    return z ** 4 / 12.0 - z ** 5 / 10.0 + z ** 6 / 30.0


def _riesz_w_antider(rho: float):
    """Antiderivative (twice) of S_rho(z) = -d^{2rho} w / d|z|^{2rho} on (0,1) (Example 4.1).

    D_L^a z^k = Gamma(k+1)/Gamma(k+1-a) z^{k-a}; summing the left and right derivatives of
    w = z^2 - 2 z^3 + z^4 and multiplying by -1/(2 cos(rho pi)) (Sec. 1) gives
    S_rho(z) = (1/cos(rho pi)) sum_k c_k [z^{k-2rho} + (1-z)^{k-2rho}] / Gamma(k+1-2rho)
    with (k, c_k) = (2, 1), (3, -6), (4, 12).  Integrating twice raises each power by 2.
    """
    cs = math.cos(rho * math.pi)
    terms = ((2, 1.0), (3, -6.0), (4, 12.0))

    def G(z):
        z = np.asarray(z, dtype=np.float64)
        zc = np.clip(z, 0.0, 1.0)
        out = np.zeros_like(zc)
        for k, ck in terms:
            e = k + 2 - 2 * rho
            out += ck * (zc ** e + (1.0 - zc) ** e) / math.gamma(e + 1.0)
        return out / cs

    return G


def _time_poly_weights(t: np.ndarray, kind: str):
    """(int_{I_n} T'(t) dt, int_{I_n} T(t) dt) for the manufactured time factor T."""
    if kind == "1+t^2":
        T = lambda s: 1.0 + s * s
        IT = lambda s: s + s ** 3 / 3.0
    elif kind == "10exp(-t)":
        T = lambda s: 10.0 * np.exp(-s)
        IT = lambda s: -10.0 * np.exp(-s)
    else:
        raise ValueError(kind)
    return T(t[1:]) - T(t[:-1]), IT(t[1:]) - IT(t[:-1]), T


def manufactured_exact(x, y, t, time_factor: str = "1+t^2"):
    """u(x,y,t) = T(t) (x-x^2)^2 (y-y^2)^2 on (0,1)^2 (Example 4.1 with time factor T)."""
    Tt = (1.0 + t * t) if time_factor == "1+t^2" else 10.0 * math.exp(-t)
    return Tt * (x - x * x) ** 2 * (y - y * y) ** 2


def manufactured_initial(nx: int, ny: int, time_factor: str = "1+t^2") -> np.ndarray:
    """Nodal interpolant psi_0^I of the manufactured solution at t = 0, shape (N_y, N_x)."""
    x = interior_nodes(nx, 0.0, 1.0)
    y = interior_nodes(ny, 0.0, 1.0)
    return manufactured_exact(x[None, :], y[:, None], 0.0, time_factor)


def manufactured_forcing(nx: int, ny: int, t: np.ndarray, beta: float, gamma: float,
                         kx: float, ky: float, time_factor: str = "1+t^2") -> Forcing:
    """Rank-3 separable load of the manufactured solution u = T(t) w(x) w(y) on (0,1)^2.

    f = T' w(x) w(y) + T [K_x S_beta(x) w(y) + K_y w(x) S_gamma(y)] (Example 4.1).
    Space integrals are exact (second differences of closed-form antiderivatives);
    time integrals are exact.
    """
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    x = interior_nodes(nx, 0.0, 1.0)
    y = interior_nodes(ny, 0.0, 1.0)
    wx = _load_second_difference(_w_antider, x, hx)
    wy = _load_second_difference(_w_antider, y, hy)
    sx = _load_second_difference(_riesz_w_antider(beta), x, hx)
    sy = _load_second_difference(_riesz_w_antider(gamma), y, hy)
    dT, iT, _ = _time_poly_weights(np.asarray(t, dtype=np.float64), time_factor)
    time_w = np.stack([dT, iT, iT], axis=1)
    bx = np.stack([wx, kx * sx, wx])
    by = np.stack([wy, wy, ky * sy])
    return Forcing(time_w, bx, by)


_GL_X, _GL_W = np.polynomial.legendre.leggauss(10)


def _hat_load_gauss(f, nodes: np.ndarray, h: float) -> np.ndarray:
    """(f, phi_i) by 10-point Gauss-Legendre on each of the two elements of the hat (smooth f)."""
    out = np.zeros_like(nodes)
    for side in (-1.0, 1.0):
        # element between x_i and x_i + side*h; hat = 1 - |z - x_i|/h
        s = 0.5 * (1.0 + _GL_X)  # in (0,1): distance fraction from x_i
        z = nodes[:, None] + side * h * s[None, :]
        out += 0.5 * h * ((1.0 - s)[None, :] * _GL_W[None, :] * f(z)).sum(axis=1)
    return out


def gaussian_bump_forcing(seed: int, nx: int, ny: int, t: np.ndarray,
                          omega=(0.0, 1.0, 0.0, 1.0)):
    """Rank-1 load of f = exp(-((x-x0)^2+(y-y0)^2)/(2 s^2)) sin(2 pi t).

    x0, y0 ~ U(0.3, 0.7) (relative to Omega) and s ~ U(0.05, 0.15), drawn with PCG64(seed).
    Returns (Forcing, (x0, y0, s)).
    """
    rng = np.random.default_rng(seed)
    x0r, y0r = rng.uniform(0.3, 0.7, size=2)
    s = float(rng.uniform(0.05, 0.15))
    a, b, c, d = omega
    x0 = a + x0r * (b - a)
    y0 = c + y0r * (d - c)
    hx, hy = (b - a) / (nx + 1), (d - c) / (ny + 1)
    x = interior_nodes(nx, a, b)
    y = interior_nodes(ny, c, d)
    bx = _hat_load_gauss(lambda z: np.exp(-(z - x0) ** 2 / (2 * s * s)), x, hx)
    by = _hat_load_gauss(lambda z: np.exp(-(z - y0) ** 2 / (2 * s * s)), y, hy)
    t = np.asarray(t, dtype=np.float64)
    tw = (np.cos(2 * np.pi * t[:-1]) - np.cos(2 * np.pi * t[1:])) / (2 * np.pi)
    return Forcing(tw[:, None].copy(), bx[None, :], by[None, :]), (x0, y0, s)


@dataclass
class DenseForcing:
    """Load vectors given slice by slice: F[n-1] = F_n, shape (N_t, N_y, N_x) (no structure)."""
    F: np.ndarray

    def dense(self, n: int) -> np.ndarray:
        """F_n as an (N_y, N_x) array (n = 1..N_t)."""
        return self.F[n - 1]


_GL5_X, _GL5_W = np.polynomial.legendre.leggauss(5)


def moving_bump_dense_forcing(seed: int, nx: int, ny: int, t: np.ndarray, speed: float | None = None,
                              omega=(0.0, 1.0, 0.0, 1.0)):
    """Non-separable load of f = exp(-((x - x0 - v t)^2 + (y - y0)^2) / (2 s^2)), a bump moving in x.

    x0, y0 ~ U(0.3, 0.7), s ~ U(0.05, 0.15) and v ~ U(-0.3, 0.3) (relative to Omega, unless ``speed``
    is given) are drawn with PCG64(seed).  F_n[j, i] = by[j] * int_{I_n} (f_x(., t), phi_i) dt with the
    space integral by 10-point Gauss-Legendre per element and the time integral by 5-point
    Gauss-Legendre per step.  Returns (DenseForcing, (x0, y0, s, v)).
    """
    rng = np.random.default_rng(seed)
    x0r, y0r = rng.uniform(0.3, 0.7, size=2)
    s = float(rng.uniform(0.05, 0.15))
    vr = float(rng.uniform(-0.3, 0.3)) if speed is None else float(speed)
    a, b, c, d = omega
    x0, y0, v = a + x0r * (b - a), c + y0r * (d - c), vr * (b - a)
    hx, hy = (b - a) / (nx + 1), (d - c) / (ny + 1)
    x = interior_nodes(nx, a, b)
    y = interior_nodes(ny, c, d)
    by = _hat_load_gauss(lambda z: np.exp(-(z - y0) ** 2 / (2 * s * s)), y, hy)
    t = np.asarray(t, dtype=np.float64)
    nt = len(t) - 1
    F = np.empty((nt, ny, nx))
    for n in range(1, nt + 1):
        lo, hi = t[n - 1], t[n]
        fx = np.zeros(nx)
        for q in range(5):
            tq = 0.5 * (lo + hi) + 0.5 * (hi - lo) * _GL5_X[q]
            cx = x0 + v * tq
            fx += 0.5 * (hi - lo) * _GL5_W[q] * _hat_load_gauss(lambda z: np.exp(-(z - cx) ** 2 / (2 * s * s)), x, hx)
        F[n - 1] = by[:, None] * fx[None, :]
    return DenseForcing(F), (x0, y0, s, v)


# ----------------------------------------------------------------------------- P1-triangle loads

@dataclass
class LowRankDenseForcing:
    """Load vectors F_n = sum_r time_w[n-1, r] G[r] with full spatial patterns G[r] of shape
    (N_y, N_x): the load of a source sum_r c_r(t) g_r(x, y) against hats that are not tensor
    products (the P1 triangles of Sec. 2)."""
    time_w: np.ndarray   # (N_t, R)
    G: np.ndarray        # (R, N_y, N_x)

    def dense(self, n: int) -> np.ndarray:
        return np.tensordot(self.time_w[n - 1], self.G, axes=1)

    def all(self) -> np.ndarray:
        """Every F_n, shape (N_t, N_y, N_x)."""
        return np.tensordot(self.time_w, self.G, axes=1)


_GL20_X, _GL20_W = np.polynomial.legendre.leggauss(20)


def _p1_hat_load(Ga, b, xa: np.ndarray, ha: float, yb: np.ndarray, hb: float) -> np.ndarray:
    """(a(x) b(y), phi_ij) for the P1 hats of the triangulation with south-west to north-east
    diagonals, result[j, i] for x_i in xa, y_j in yb; Ga is a second antiderivative of a (Ga'' = a).

    In local coordinates s = (x - x_i)/h_a, r = (y - y_j)/h_b the hat is max(0, 1 - max(|s|, |r|, |s - r|)).
    At fixed r it is, in s, a trapezoid with kinks at r - 1, 0, r, 1 (r > 0) or -1, r, 0, 1 + r (r < 0),
    so its integral against a is exact by two integrations by parts (sum over the kinks of the slope
    jump times Ga).  The remaining integral over r is a 20-point Gauss-Legendre rule on (-1, 0) and on
    (0, 1), with b evaluated along the r direction (b smooth in the cases used here).
    """
    out = np.zeros((len(yb), len(xa)))
    for lo in (-1.0, 0.0):
        r = lo + 0.5 * (_GL20_X + 1.0)
        w = 0.5 * _GL20_W
        X = xa[:, None]
        R = r[None, :]
        if lo == 0.0:
            J = (Ga(X + (R - 1.0) * ha) - Ga(X) - Ga(X + R * ha) + Ga(X + ha)) / ha
        else:
            J = (Ga(X - ha) - Ga(X + R * ha) - Ga(X) + Ga(X + (1.0 + R) * ha)) / ha
        B = b(yb[:, None] + r[None, :] * hb)
        out += hb * (B * w[None, :]) @ J.T
    return out


def _w(z):
    return (z - z * z) ** 2


def p1_manufactured_forcing(nx: int, ny: int, t: np.ndarray, beta: float, gamma: float, kx: float, ky: float,
                            time_factor: str = "10exp(-t)") -> LowRankDenseForcing:
    """Load vectors of the manufactured solution u = T(t) w(x) w(y) (Example 4.1, T = 10 e^{-t}) against
    the P1 hats: f = T' w(x) w(y) + T [K_x S_beta(x) w(y) + K_y w(x) S_gamma(y)].  Every term is a product
    a(x) b(y); the factor with the weak boundary singularity (S_rho, the Riesz derivative of w) is
    integrated exactly in its own direction (``_p1_hat_load``), the smooth one by Gauss-Legendre.  Time
    integrals are exact.  Domain (0, 1)^2."""
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    x = interior_nodes(nx, 0.0, 1.0)
    y = interior_nodes(ny, 0.0, 1.0)
    L_ww = _p1_hat_load(_w_antider, _w, x, hx, y, hy)
    L_sw = _p1_hat_load(_riesz_w_antider(beta), _w, x, hx, y, hy)
    L_ws = _p1_hat_load(_riesz_w_antider(gamma), _w, y, hy, x, hx).T   # singular factor in y
    dT, iT, _ = _time_poly_weights(np.asarray(t, dtype=np.float64), time_factor)
    return LowRankDenseForcing(np.stack([dT, iT, iT], axis=1), np.stack([L_ww, kx * L_sw, ky * L_ws]))


# ----------------------------------------------------------------------------- workloads

@dataclass
class Workload:
    """One SFDE instance plus the MGRIT settings it is solved with."""
    name: str
    beta: float
    gamma: float
    kx: float
    ky: float
    nx: int
    ny: int
    nt: int
    m: int
    omega: tuple = (0.0, 1.0, 0.0, 1.0)
    T: float = 1.0
    grid: str = "uniform"
    psi0: str = "sine"          # "sine" | "manufactured"
    source: str = "zero"        # "zero" | "manufactured" | "bump"
    max_levels: int = 32
    rel_tol: float = 1e-10
    seed: int = 0
    notes: str = ""
    _cache: dict = field(default_factory=dict, repr=False)

    def t(self) -> np.ndarray:
        return time_grid(self.nt, self.T, self.grid)

    def initial(self) -> np.ndarray:
        if self.psi0 == "manufactured":
            return manufactured_initial(self.nx, self.ny)
        return sine_mode_nodal(sine_mode_amplitudes(self.seed), self.nx, self.ny, self.omega)

    def forcing(self) -> Optional[Forcing]:
        if self.source == "zero":
            return None
        if self.source == "manufactured":
            return manufactured_forcing(self.nx, self.ny, self.t(), self.beta, self.gamma,
                                        self.kx, self.ky)
        if self.source == "bump":
            return gaussian_bump_forcing(self.seed + 1, self.nx, self.ny, self.t(), self.omega)[0]
        raise ValueError(self.source)

    @property
    def dofs(self) -> int:
        return self.nx * self.ny

    @property
    def space_time_updates(self) -> int:
        return self.nx * self.ny * self.nt


WORKLOADS = {
    # manufactured solution u = (1+t^2) x^2(1-x)^2 y^2(1-y)^2, two-level MGRIT, m = 4
    "manufactured_N31_Nt64": Workload(
        "manufactured_N31_Nt64", 0.75, 0.75, 1.0, 1.0, 31, 31, 64, 4,
        psi0="manufactured", source="manufactured", max_levels=2),
    # 16 seeded sine modes, f = 0, multilevel V-cycle, m = 8
    "sine_N255_Nt1024": Workload(
        "sine_N255_Nt1024", 0.6, 0.9, 1.0, 0.5, 255, 255, 1024, 8),
    # strong anisotropy, Gaussian bump x sin(2 pi t)
    "bump_N511_Nt2048": Workload(
        "bump_N511_Nt2048", 0.55, 0.95, 1.0, 0.1, 511, 511, 2048, 8, source="bump", rel_tol=1e-8),
    # graded time grid t_n = (n/N)^2, m = 16
    "graded_N1023_Nt4096": Workload(
        "graded_N1023_Nt4096", 0.7, 0.8, 1.0, 1.0, 1023, 1023, 4096, 16, grid="graded",
        source="bump", rel_tol=1e-8),
}


def batch_workloads(seed: int = 0, count: int = 64) -> list[Workload]:
    """Uneven batch: N in {63,127,255,511}, N_t in {256,512,1024,4096}, beta, gamma ~ U(0.55,0.95),
    K_x, K_y ~ U[0.1, 2], all drawn with PCG64(seed); sine-mode psi_0 (seed 1000+k), f = 0, m = 8."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.choice([63, 127, 255, 511]))
        nt = int(rng.choice([256, 512, 1024, 4096]))
        b, g = rng.uniform(0.55, 0.95, size=2)
        kx, ky = rng.uniform(0.1, 2.0, size=2)
        out.append(Workload(f"batch{k}_N{n}_Nt{nt}", float(b), float(g), float(kx), float(ky),
                            n, n, nt, 8, seed=1000 + k, rel_tol=1e-8))
    return out


def workload(name: str) -> Workload:
    return WORKLOADS[name]

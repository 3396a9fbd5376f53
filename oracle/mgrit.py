"""MGRIT (Algorithm 1) for the block bidiagonal system of Eq. (3.1) -- FP64 CPU oracle.

Test infrastructure only.  Two executions of the same algorithm:

* ``mgrit``        -- nodal coordinates, one call of ``SFDE.step``/``SFDE.propagate`` per
                      time step (the plain statement of Algorithm 1);
* ``mgrit_modal``  -- the same iteration carried out in the basis that diagonalises every
                      propagator at once (Eqs. (3.5)-(3.7)); it produces the same iterates up to
                      rounding at O(N^2) cost per step and is pinned against ``mgrit``.

Algorithm 1 with the readings used throughout this project:

* level l has the time grid t^(l), t^(l+1)_k = t^(l)_{km} (Sec. 3.1); levels are added while
  N_l is divisible by m and N_l/m >= min_coarse, up to max_levels;
* level-0 step Phi_n(u) = Psi_n u + g_n = S_n^{-1}(B_n u + F_n) (Eqs. (2.4), (3.1), (3.2));
* coarse steps Phi^(l)_k(v) = Psi^Delta_k v + g^(l)_k with Psi^Delta the rediscretisation of
  Eq. (3.4) ("cn", the paper's choice) or the L-stable backward-Euler rediscretisation ("be");
  the fixed point of the iteration does not depend on this choice;
* Step 1: FCF relaxation (Sec. 3.1; "F" relaxation gives the parareal-type variant);
* Step 2: injection of the C-point residual r_k = Phi_{km}(u_{km-1}) - u_{km}, r_0 = g_0 - u_0;
* Step 3: recursion with zero initial guess; the coarsest level is solved by sequential stepping;
* Step 4: correction at C-points only; on levels l >= 1 the interpolation is injection followed by
  an F-relaxation; on level 0 F-points are refreshed by the next iteration's relaxation
  (the remark after Algorithm 1);
* stopping: ||r||_2 over all level-0 C-points <= max(rel_tol * ||r^(first)||_2, abs_tol), tested
  right after the level-0 residual (so the returned iterate is F-consistent); or (stop="sform")
  the norm of the space-time residual rho_n = F_n + B_n u_{n-1} - S_n u_n over n = 1..N_t (the rows
  of Eq. (3.1) multiplied by S_n), relative to that of the initial guess, tested at the same place;
* skip_first_down (the option of Sec. 3.2): on the first iteration the down-cycle does no
  relaxation on any level -- the coarse right-hand side is the injected C-point residual of the
  initial guess (on levels >= 1, whose guess is zero, that is the injected right-hand side) -- and
  the coarsest solve and the up-cycle run as usual; that iteration applies no stopping test, and the
  C-point reference norm is the second iteration's.
"""
from __future__ import annotations

import numpy as np

from .sfde import SFDE, modal_lambda

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_uniform(seed: int, start: int, count: int) -> np.ndarray:
    """Counter-based uniform[-1,1) values from the SplitMix64 finaliser (Steele, Lea, Flood 2014).

    SplitMix64 advances its state by phi = 0x9E3779B97F4A7C15 and mixes it; output number idx
    (0-based) of the generator seeded with ``seed`` is mix(seed + (idx+1) phi), all mod 2^64.
    value(idx) = 2 * (mix(...) >> 11) * 2^-53 - 1; ``idx`` runs over start .. start+count-1.
    """
    with np.errstate(over="ignore"):
        idx = np.arange(start, start + count, dtype=np.uint64)
        z = np.uint64(seed) + (idx + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def initial_guess(U0, nt: int, init_seed: int = 0):
    """u_0 = psi_0^I; u_n = 0 (init_seed = 0) or SplitMix64 uniform[-1,1) values (Sec. 3.2 choice
    of random initial guesses), index (n*N_y + j)*N_x + i."""
    ny, nx = U0.shape
    u = np.zeros((nt + 1, ny, nx))
    u[0] = U0
    if init_seed:
        u[1:] = splitmix64_uniform(init_seed, ny * nx, nt * ny * nx).reshape(nt, ny, nx)
    return u


def build_levels(t: np.ndarray, m: int, max_levels: int = 32, min_coarse: int = 2):
    """Time grids of the hierarchy: t^(0) = t, t^(l+1) = t^(l)[::m]."""
    if m < 2:
        raise ValueError("coarsening factor m must be >= 2")
    levels = [np.asarray(t, dtype=np.float64)]
    while (len(levels) < max_levels and (len(levels[-1]) - 1) % m == 0
           and (len(levels[-1]) - 1) // m >= min_coarse):
        levels.append(levels[-1][::m].copy())
    return levels


class MGRITResult:
    def __init__(self, U, history, iters, levels, converged, step_solves):
        self.U = U
        self.history = history
        self.iters = iters
        self.levels = levels
        self.converged = converged
        self.step_solves = step_solves

    @property
    def conv_factor_last5(self):
        h = self.history
        if len(h) < 2:
            return float("nan")
        r = [h[i + 1] / h[i] for i in range(len(h) - 1) if h[i] > 0]
        r = r[-5:]
        return float(np.mean(r)) if r else float("nan")


def space_time_residual(prob: SFDE, U, forcing=None):
    """rho_n = F_n + B_n U_{n-1} - S_n U_n, n = 1..N_t: the residual of the fully discrete scheme
    Eq. (2.4) at every time point (row n of the block system Eq. (3.1), multiplied by S_n).
    Returns an (N_t, N_y, N_x) array."""
    U = np.asarray(U, dtype=np.float64)
    out = np.empty((prob.nt,) + U.shape[1:])
    for n in range(1, prob.nt + 1):
        tau = 0.5 * (prob.t[n] - prob.t[n - 1])
        r = prob.apply_B(U[n - 1], tau) - prob.apply_S(U[n], tau)
        if forcing is not None:
            r = r + forcing.dense(n)
        out[n - 1] = r
    return out


def mgrit(prob: SFDE, U0, forcing=None, m: int = 2, max_levels: int = 32, min_coarse: int = 2,
          coarse: str = "cn", relax: str = "FCF", rel_tol: float = 1e-10, abs_tol: float = 0.0,
          max_iter: int = 100, init_seed: int = 0, dense: bool = False, skip_first_down: bool = False,
          stop: str = "cpoint") -> MGRITResult:
    """Algorithm 1 in nodal coordinates.  Returns all time points U[0..N_t]."""
    if stop not in ("cpoint", "sform"):
        raise ValueError(stop)
    levels = build_levels(prob.t, m, max_levels, min_coarse)
    L = len(levels)
    counter = [0]

    def phi(l, n, v, g):
        counter[0] += 1
        if l == 0:
            F = None if forcing is None else forcing.dense(n)
            return prob.step(v, n, F, dense=dense)
        dt = levels[l][n] - levels[l][n - 1]
        return prob.propagate(v, dt, coarse, dense=dense) + g[n]

    def frelax(l, u, g):
        N = len(levels[l]) - 1
        for n in range(1, N + 1):
            if n % m:
                u[n] = phi(l, n, u[n - 1], g)

    def crelax(l, u, g):
        N = len(levels[l]) - 1
        for n in range(m, N + 1, m):
            u[n] = phi(l, n, u[n - 1], g)

    def relaxation(l, u, g):
        frelax(l, u, g)
        if relax == "FCF":
            crelax(l, u, g)
            frelax(l, u, g)
        elif relax != "F":
            raise ValueError(relax)

    def residual(l, u, g):
        N = len(levels[l]) - 1
        r = np.zeros((N // m + 1,) + u.shape[1:])
        r[0] = (g[0] - u[0]) if l > 0 else 0.0  # u_0 = psi_0 exactly on level 0
        for k in range(1, N // m + 1):
            r[k] = phi(l, k * m, u[k * m - 1], g) - u[k * m]
        return r

    def solve(l, u, g, skip=False):
        """Approximately solve the level-l system (recursive part of Algorithm 1); with skip the
        down-cycle does no relaxation."""
        N = len(levels[l]) - 1
        if l == L - 1:
            u[0] = g[0]
            for n in range(1, N + 1):
                u[n] = phi(l, n, u[n - 1], g)
            return
        if not skip:
            relaxation(l, u, g)
        r = residual(l, u, g)
        v = np.zeros_like(r)
        solve(l + 1, v, r, skip)
        u[::m] += v
        frelax(l, u, g)

    def sform_norm(u):
        rho = space_time_residual(prob, u, forcing)
        return float(np.sqrt(np.sum(rho * rho)))

    u = initial_guess(np.asarray(U0, dtype=np.float64), prob.nt, init_seed)
    if L == 1:
        solve(0, u, u[:1])
        return MGRITResult(u, [0.0], 1, 1, True, counter[0])
    hist = []
    ref = sform_norm(u) if stop == "sform" else None
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        skip = skip_first_down and it == 1
        if not skip:
            relaxation(0, u, None)
        r = residual(0, u, None)
        nrm = sform_norm(u) if stop == "sform" else float(np.sqrt(np.sum(r * r)))
        hist.append(nrm)
        if not np.isfinite(nrm):
            break
        # a skipped iteration's residual is that of the unrelaxed guess: no stopping test there, and
        # the C-point reference is the first norm computed after a relaxation
        if not skip:
            first = ref if stop == "sform" else hist[1 if skip_first_down else 0]
            if nrm <= max(rel_tol * first, abs_tol):
                converged = True
                break
        v = np.zeros_like(r)
        solve(1, v, r, skip)
        u[::m] += v
    return MGRITResult(u, hist, it, L, converged, counter[0])


def mgrit_modal(prob: SFDE, U0, forcing=None, m: int = 2, max_levels: int = 32,
                min_coarse: int = 2, coarse: str = "cn", relax: str = "FCF",
                rel_tol: float = 1e-10, abs_tol: float = 0.0, max_iter: int = 100,
                init_seed: int = 0, keep_all: bool = False) -> MGRITResult:
    """Algorithm 1 carried out on modal coefficients c = W_y^T u W_x (W = M V), where every
    propagator is diagonal (Eq. (3.6)): Psi_n -> lambda_n (Eq. (3.7)), Psi^Delta -> mu_k.
    Residual norms are measured in nodal coordinates (r = V_y r_hat V_x^T), so the history is
    directly comparable with ``mgrit``.  Returns U[N_t] only unless keep_all."""
    lx, Vx, ly, Vy = prob.eig()
    sig = prob.sigma()
    Wx, Wy = prob.Mx @ Vx, prob.My @ Vy
    levels = build_levels(prob.t, m, max_levels, min_coarse)
    L = len(levels)
    dts = [np.diff(tl) for tl in levels]
    if forcing is not None:
        px = forcing.bx @ Vx
        py = forcing.by @ Vy
    counter = [0]

    def step_many(l, idx, v, g):
        """Apply Phi^(l)_n for every n in idx (array) to v (len(idx), N_y, N_x)."""
        counter[0] += len(idx)
        dt = dts[l][idx - 1][:, None, None]
        if l == 0:
            out = modal_lambda(sig[None], dt, "cn") * v
            if forcing is not None:
                fh = np.einsum("nr,rj,ri->nji", forcing.time_w[idx - 1], py, px)
                out += fh / (1.0 + 0.5 * dt * sig[None])
            return out
        return modal_lambda(sig[None], dt, coarse) * v + g[idx]

    def frelax(l, c, g):
        N = len(levels[l]) - 1
        for j in range(1, m):
            idx = np.arange(j, N + 1, m)
            if len(idx):
                c[idx] = step_many(l, idx, c[idx - 1], g)

    def crelax(l, c, g):
        N = len(levels[l]) - 1
        idx = np.arange(m, N + 1, m)
        c[idx] = step_many(l, idx, c[idx - 1], g)

    def relaxation(l, c, g):
        frelax(l, c, g)
        if relax == "FCF":
            crelax(l, c, g)
            frelax(l, c, g)

    def residual(l, c, g):
        N = len(levels[l]) - 1
        idx = np.arange(m, N + 1, m)
        r = np.zeros((N // m + 1,) + c.shape[1:])
        r[0] = (g[0] - c[0]) if l > 0 else 0.0
        r[1:] = step_many(l, idx, c[idx - 1], g) - c[idx]
        return r

    def solve(l, c, g):
        N = len(levels[l]) - 1
        if l == L - 1:
            c[0] = g[0]
            for n in range(1, N + 1):
                c[n] = step_many(l, np.array([n]), c[n - 1:n], g)[0]
            return
        relaxation(l, c, g)
        r = residual(l, c, g)
        v = np.zeros_like(r)
        solve(l + 1, v, r)
        c[::m] += v
        frelax(l, c, g)

    u0 = initial_guess(np.asarray(U0, dtype=np.float64), prob.nt, init_seed)
    c = np.einsum("jb,nji,ia->nba", Wy, u0, Wx) if init_seed else np.zeros_like(u0)
    if not init_seed:
        c[0] = Wy.T @ u0[0] @ Wx
    del u0
    hist = []
    converged = False
    it = 0
    if L == 1:
        solve(0, c, c[:1])
        it, converged, hist = 1, True, [0.0]
    else:
        for it in range(1, max_iter + 1):
            relaxation(0, c, None)
            r = residual(0, c, None)
            nrm = float(np.sqrt(sum(np.sum((Vy @ rk @ Vx.T) ** 2) for rk in r)))
            hist.append(nrm)
            if nrm <= max(rel_tol * hist[0], abs_tol) or not np.isfinite(nrm):
                converged = bool(np.isfinite(nrm))
                break
            v = np.zeros_like(r)
            solve(1, v, r)
            c[::m] += v
    if keep_all:
        U = np.einsum("jb,nba,ia->nji", Vy, c, Vx)
    else:
        U = Vy @ c[-1] @ Vx.T
    return MGRITResult(U, hist, it, L, converged, counter[0])

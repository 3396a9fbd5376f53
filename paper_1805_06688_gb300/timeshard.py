"""Time-sharded MGRIT: Algorithm 1 (Sec. 3.1) with the time axis split across ranks, one rank per GPU
(the paper's temporal communicator, Sec. 3.2).

Partition.  Level 0 has N_t / m coarse intervals; with R ranks, rank r owns a contiguous block of
N_t / (m R) of them, i.e. the time points (lo, hi] = (r N_t / R, (r + 1) N_t / R].  Level l + 1's points
are level l's C-points, so rank r owns the level-(l + 1) points (lo / m, hi / m].  A level is relaxed
across the ranks while every rank's share is a whole number (>= 1) of its intervals and the level is
not the coarsest; the first level where that fails is gathered (one all-gather of its right-hand
side) and every rank solves it and the levels below it the same way, keeping the correction of its
own points.

Messages of one V-cycle, per distributed level: before each F-relaxation every rank sends its last
point to the next rank (the ghost point lo of that rank: one slice per boundary); the C-point residual
norm of the fine level is one scalar all-reduce per iteration; the gathered level is one all-gather.
The iteration is the library's FP64 V-cycle (mgrit_solve with SFDE_PREC_FP64, C-point residual
stopping test, no final F-relaxation on the fine level), so with the same steps its iterates equal the
single-rank ones up to the order of the norm's sum.

The steps are callbacks (a Stepper), so the message logic is independent of where the steps run:
LibraryStepper applies them with the GPU library (sfde_step_batch / sfde_propagate_batch); tests plug
in other step implementations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch
import torch.distributed as dist

from . import _binding as B


class Stepper:
    """Step callbacks on torch tensors of shape (batch, N_y, N_x).

    fine(n0, dn, V):   Phi_{n0 + b dn}(V_b) = S_n^{-1}(B_n V_b + F_n), the fine step of Eq. (2.4);
    coarse(dts, V, G): Psi(dts[b]) V_b + G_b (G may be None), the coarse propagator (Eq. (3.4), or
                       the backward-Euler rediscretisation) with a right-hand side.
    """

    def fine(self, n0: int, dn: int, V: torch.Tensor) -> torch.Tensor:  # pragma: no cover - protocol
        raise NotImplementedError

    def coarse(self, dts, V: torch.Tensor, G) -> torch.Tensor:  # pragma: no cover - protocol
        raise NotImplementedError


class LibraryStepper(Stepper):
    """The steps of a Problem (FP64) on the GPU: sfde_step_batch and sfde_propagate_batch."""

    def __init__(self, problem, coarse=B.COARSE_BE):
        if coarse not in (B.COARSE_CN, B.COARSE_BE):
            raise ValueError("coarse propagator must be COARSE_CN or COARSE_BE")
        self.P = problem
        self.scheme = coarse

    def fine(self, n0, dn, V):
        out = torch.empty_like(V)
        B.sfde_step_batch(self.P.ctx, n0, dn, V.shape[0], V.contiguous(), out)
        return out

    def coarse(self, dts, V, G):
        out = torch.empty_like(V)
        B.sfde_propagate_batch(self.P.ctx, self.scheme, np.asarray(dts, dtype=np.float64), V.contiguous(), out,
                               None if G is None else G.contiguous())
        return out


@dataclass
class ShardedResult:
    U: torch.Tensor          # this rank's points lo..hi of the fine level (index 0: point lo)
    lo: int
    hi: int
    history: list = field(default_factory=list)
    iters: int = 0
    converged: bool = False
    distributed_levels: int = 0
    levels: int = 0


def level_sizes(nt: int, m: int, max_levels: int, min_coarse: int):
    """Points per level: coarsen by m while the level divides, keeps >= min_coarse coarse points
    and max_levels allows it (the rule of the library's FP64 hierarchy)."""
    n = [nt]
    while len(n) < max_levels and n[-1] % m == 0 and n[-1] // m >= min_coarse:
        n.append(n[-1] // m)
    return n


class _Comm:
    def __init__(self, group):
        self.group = group
        self.R = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
        self.r = dist.get_rank(group) if self.R > 1 else 0

    def ghost(self, u: torch.Tensor):
        """u[0] <- the previous rank's last point (its u[-1])."""
        if self.R == 1:
            return
        reqs, buf = [], None
        if self.r + 1 < self.R:
            reqs.append(dist.isend(u[-1].contiguous(), self.r + 1, group=self.group))
        if self.r > 0:
            buf = torch.empty_like(u[0])
            reqs.append(dist.irecv(buf, self.r - 1, group=self.group))
        for q in reqs:
            q.wait()
        if buf is not None:
            u[0] = buf

    def sum(self, x: float, device) -> float:
        if self.R == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return float(t.item())

    def gather(self, own: torch.Tensor) -> torch.Tensor:
        if self.R == 1:
            return own
        parts = [torch.empty_like(own) for _ in range(self.R)]
        dist.all_gather(parts, own.contiguous(), group=self.group)
        return torch.cat(parts)


def time_sharded_mgrit(stepper: Stepper, t, psi0: torch.Tensor, m: int, max_levels: int = 32, min_coarse: int = 2,
                       relax: str = "FCF", rel_tol: float = 1e-10, abs_tol: float = 0.0, max_iter: int = 100,
                       group=None) -> ShardedResult:
    """Algorithm 1 on R ranks (the torch.distributed group `group`, or the default one; a single process
    without an initialised group is R = 1).  t: the fine time grid (host, N_t + 1 values, the same on
    every rank); psi0: the initial values (N_y, N_x).  Returns this rank's fine-level points."""
    if relax not in ("FCF", "F"):
        raise ValueError(relax)
    comm = _Comm(group)
    R, r = comm.R, comm.r
    t = np.asarray(t, dtype=np.float64)
    nt = len(t) - 1
    if m < 2:
        raise ValueError("m must be >= 2")
    sizes = level_sizes(nt, m, max_levels, min_coarse)
    L = len(sizes)
    grids = [t[:: m ** l] for l in range(L)]
    dts = [np.diff(g) for g in grids]
    dev = psi0.device
    shape = tuple(psi0.shape)

    # distributed levels: every rank holds whole intervals, and the level is not the coarsest
    Ld = 0
    while Ld < L - 1 and sizes[Ld] % R == 0 and (sizes[Ld] // R) % m == 0 and sizes[Ld] // R >= m:
        Ld += 1

    def zeros(k):
        return torch.zeros((k,) + shape, dtype=torch.float64, device=dev)

    def ix(a):
        return torch.as_tensor(np.asarray(a), dtype=torch.long, device=dev)

    def phi(l, n0, dn, V, G):
        """level-l steps to the points n0 + b dn (global indices of the level)."""
        if l == 0:
            return stepper.fine(n0, dn, V)
        idx = n0 + dn * np.arange(V.shape[0])
        return stepper.coarse(dts[l][idx - 1], V, G)

    # ---------------------------------------------------------------- serial part (full levels)
    def s_frelax(l, u, g):
        for j in range(1, m):
            idx = np.arange(j, sizes[l] + 1, m)
            if len(idx):
                u[ix(idx)] = phi(l, j, m, u[ix(idx - 1)], None if g is None else g[ix(idx)])

    def s_crelax(l, u, g):
        idx = np.arange(m, sizes[l] + 1, m)
        u[ix(idx)] = phi(l, m, m, u[ix(idx - 1)], None if g is None else g[ix(idx)])

    def s_relax(l, u, g):
        s_frelax(l, u, g)
        if relax == "FCF":
            s_crelax(l, u, g)
            s_frelax(l, u, g)

    def s_residual(l, u, g):
        idx = np.arange(m, sizes[l] + 1, m)
        res = zeros(len(idx) + 1)
        if l > 0:
            res[0] = g[0] - u[0]
        res[1:] = phi(l, m, m, u[ix(idx - 1)], None if g is None else g[ix(idx)]) - u[ix(idx)]
        return res

    def s_solve(l, u, g):
        if l == L - 1:
            u[0] = g[0]
            for n in range(1, sizes[l] + 1):
                u[n] = phi(l, n, 1, u[n - 1:n], g[n:n + 1])[0]
            return
        s_relax(l, u, g)
        res = s_residual(l, u, g)
        v = zeros(sizes[l + 1] + 1)
        s_solve(l + 1, v, res)
        u[::m] += v
        s_frelax(l, u, g)

    # ---------------------------------------------------------------- distributed levels
    lo = [r * sizes[l] // R for l in range(L)]
    hi = [(r + 1) * sizes[l] // R for l in range(L)]

    def d_frelax(l, u, g):
        comm.ghost(u)
        for j in range(1, m):
            k = np.arange(0, hi[l] - lo[l], m) + j          # local indices of the j-th F-points
            u[ix(k)] = phi(l, lo[l] + j, m, u[ix(k - 1)], None if g is None else g[ix(k)])

    def d_crelax(l, u, g):
        k = np.arange(m, hi[l] - lo[l] + 1, m)
        u[ix(k)] = phi(l, lo[l] + m, m, u[ix(k - 1)], None if g is None else g[ix(k)])

    def d_relax(l, u, g):
        d_frelax(l, u, g)
        if relax == "FCF":
            d_crelax(l, u, g)
            d_frelax(l, u, g)

    def d_residual(l, u, g):
        """the level-(l + 1) right-hand side at this rank's coarse points (local array with ghost 0)
        and this rank's sum of squares of the C-point residuals"""
        k = np.arange(m, hi[l] - lo[l] + 1, m)
        res = zeros(len(k) + 1)
        rk = phi(l, lo[l] + m, m, u[ix(k - 1)], None if g is None else g[ix(k)]) - u[ix(k)]
        res[1:] = rk
        return res, float((rk * rk).sum().item())

    def d_solve(l, g):
        """approximate solution of the level-l correction system, zero initial guess: this rank's
        points lo..hi (index 0 the ghost, zero for rank 0)"""
        if l >= Ld:
            full = zeros(sizes[l] + 1)
            full[1:] = comm.gather(g[1:])           # point 0 of a coarse level carries no right-hand side
            v = zeros(sizes[l] + 1)
            s_solve(l, v, full)
            return v[lo[l]: hi[l] + 1].clone()
        u = zeros(hi[l] - lo[l] + 1)
        d_relax(l, u, g)
        res, _ = d_residual(l, u, g)
        v = d_solve(l + 1, res)
        u[m::m] += v[1:]
        d_frelax(l, u, g)
        return u

    # ---------------------------------------------------------------- iteration on the fine level
    if Ld == 0:
        # nothing to split: every rank runs the whole iteration and keeps its own points
        u = zeros(nt + 1)
        u[0] = psi0
        hist, it, conv = [], 0, False
        if L == 1:   # no coarse level: sequential stepping
            for n in range(1, nt + 1):
                u[n] = phi(0, n, 1, u[n - 1:n], None)[0]
            return ShardedResult(u[lo[0]: hi[0] + 1].clone(), lo[0], hi[0], [0.0], 1, True, 0, L)
        for it in range(1, max_iter + 1):
            s_relax(0, u, None)
            res = s_residual(0, u, None)
            nrm = math.sqrt(float((res[1:] * res[1:]).sum().item()))
            hist.append(nrm)
            if not math.isfinite(nrm):
                break
            if nrm <= max(rel_tol * hist[0], abs_tol):
                conv = True
                break
            v = zeros(sizes[1] + 1)
            s_solve(1, v, res)
            u[::m] += v
        return ShardedResult(u[lo[0]: hi[0] + 1].clone(), lo[0], hi[0], hist, it, conv, 0, L)

    u = zeros(hi[0] - lo[0] + 1)
    if r == 0:
        u[0] = psi0
    hist, it, conv = [], 0, False
    for it in range(1, max_iter + 1):
        d_relax(0, u, None)
        res, sq = d_residual(0, u, None)
        nrm = math.sqrt(comm.sum(sq, dev))
        hist.append(nrm)
        if not math.isfinite(nrm):
            break
        if nrm <= max(rel_tol * hist[0], abs_tol):
            conv = True
            break
        v = d_solve(1, res)
        u[m::m] += v[1:]
    return ShardedResult(u, lo[0], hi[0], hist, it, conv, Ld, L)

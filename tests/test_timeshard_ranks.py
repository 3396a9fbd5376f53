"""Time-sharded MGRIT (paper_1805_06688_gb300.timeshard) on CPU ranks (gloo): the message logic --
ghost slices before each F-relaxation, the all-reduced residual norm, the gathered coarse level --
gives the oracle's single-process Algorithm 1, iteration by iteration.  The steps are the oracle's
(a Stepper built on it), so only the partition and the messages are under test."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(nt):
    from oracle import sfde as osfde
    from sfde_workloads import gaussian_bump_forcing, sine_mode_amplitudes, sine_mode_nodal, time_grid
    nx, ny = 6, 5
    t = time_grid(nt, 1.0, "graded")
    O = osfde.SFDE(0.7, 0.85, 1.1, 0.6, nx, ny, t)
    F, _ = gaussian_bump_forcing(2, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(3), nx, ny)
    return O, F, psi, t


def _stepper(O, F, coarse):
    from paper_1805_06688_gb300.timeshard import Stepper

    class OracleStepper(Stepper):
        def fine(self, n0, dn, V):
            return torch.from_numpy(np.stack([O.step(V[b].numpy(), n0 + b * dn, F.dense(n0 + b * dn))
                                              for b in range(V.shape[0])]))

        def coarse(self, dts, V, G):
            out = [O.propagate(V[b].numpy(), dts[b], coarse) for b in range(V.shape[0])]
            if G is not None:
                out = [o + G[b].numpy() for b, o in enumerate(out)]
            return torch.from_numpy(np.stack(out))

    return OracleStepper()


def _rank_main(rank, world, port, nt, m, relax, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1805_06688_gb300.timeshard import time_sharded_mgrit
    O, F, psi, t = _problem(nt)
    res = time_sharded_mgrit(_stepper(O, F, "be"), t, torch.from_numpy(psi), m, relax=relax, rel_tol=1e-11,
                             max_iter=60)
    q.put((rank, res.lo, res.hi, res.U.numpy(), res.history, res.iters, res.converged, res.distributed_levels,
           res.levels))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,nt,m,relax,dlev", [
    (2, 64, 4, "FCF", 2),     # levels 64, 16, 4: two distributed, the coarsest gathered
    (2, 48, 4, "FCF", 1),     # 48, 12, 3: level 1 (6 points per rank) gathered and solved by every rank
    (3, 48, 4, "FCF", 2),
    (4, 32, 2, "F", 3),       # parareal-type F-relaxation, five levels
    (2, 20, 4, "FCF", 0),     # 10 points per rank is no whole number of intervals: nothing split
])
def test_time_sharded_mgrit_equals_single_process(world, nt, m, relax, dlev):
    import multiprocessing as mp
    sys.path.insert(0, ROOT)
    from oracle import mgrit as omgrit
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, nt, m, relax, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    O, F, psi, t = _problem(nt)
    ref = omgrit.mgrit(O, psi, F, m=m, coarse="be", relax=relax, rel_tol=1e-11, max_iter=60)
    U = np.zeros_like(ref.U)
    for rank, lo, hi, Ul, hist, iters, conv, Ld, L in out:
        assert conv and iters == ref.iters and L == ref.levels and Ld == dlev, (rank, iters, ref.iters, Ld)
        for a, b in zip(hist, ref.history):
            assert abs(a - b) <= 1e-12 * ref.history[0]
        U[lo:hi + 1] = Ul
    # the ranks' blocks cover the time axis; rank 0 also holds point 0 = psi_0
    assert [o[1] for o in out] == [r * nt // world for r in range(world)]
    assert np.abs(U - ref.U).max() <= 1e-12 * np.abs(ref.U).max()

"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): the whole-job throughput is
the units of all ranks over the slowest rank's time, every rank sees the same figures, and the
reference arm runs on rank 0 only (the other ranks exit 0 without output)."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r: (r + 1) seconds for 10 (r + 1) units
    rate, sec = bench.whole_job_rate(float(rank + 1), 10.0 * (rank + 1), world, "cpu")
    q.put((rank, rate, sec))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    # units 10 + 20 over the slowest rank's 2 s, on both ranks
    assert [r for r, _, _ in res] == [0, 1]
    for _, rate, sec in res:
        assert sec == 2.0 and rate == 15.0


def test_whole_job_rate_one_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(2.0, 10.0, 1) == (5.0, 2.0)


def test_reference_arm_on_other_ranks_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""

"""CPU test of the multi-rank path of bench.py (world size 2, gloo): replicas
solve their own seeded workloads and the whole-job rate is the units of all
ranks over the slowest rank's time, the same on every rank."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist                 # noqa: E402
import torch.multiprocessing as mp               # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 * (rank + 1)                # rank 1 is the slower replica
    rate, ms = bench.job_rate(local_ms, 50, world, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, rate, ms, bench.replica_seed(1, rank)))


def test_two_replicas_report_the_job_rate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    # MAX over ranks: 200 ms; units of both ranks: 2 x 50
    for _, rate, ms, _ in got:
        assert ms == 200.0
        assert rate == pytest.approx(100 / 0.2)
    assert got[0][3] != got[1][3]                # each replica its own workload

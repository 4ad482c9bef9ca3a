"""Multi-rank logic of bench.py on the CPU: two gloo ranks (world size 2,
rendezvous on 127.0.0.1) run the weak-scaling aggregation. Each rank
processes its own batch (no data-path collective); the job time is the
maximum over ranks and the value counts the units of all ranks."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 180.0][rank]
    value, max_ms = bench.job_throughput(local_ms, units_per_rank=1000, steps=10)
    env = bench.dist_env()
    out.put((rank, value, max_ms, env))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    torch = pytest.importorskip("torch")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, max_ms, env in res:
        assert max_ms == 180.0                       # slowest rank
        assert abs(value - 2 * 1000 * 10 / 0.18) < 1e-6   # all units / max time
        assert env == (2, rank, rank)


def test_single_process_throughput():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    value, max_ms = bench.job_throughput(50.0, units_per_rank=200, steps=5)
    assert max_ms == 50.0 and abs(value - 200 * 5 / 0.05) < 1e-9

"""The N > 1 bench path on CPU: two gloo ranks, replicas only (no data-path collective);
job time is the max over ranks and the job value counts every rank's work."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 * (rank + 1)                 # rank 1 is the slower replica
    tmax = bench.reduce_max(ms, world)
    val = bench.job_value(1000, 2, world, tmax)
    q.put((rank, tmax, val))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, val in res:
        assert tmax == 200.0
        assert val == pytest.approx(1000 * 2 * 2 / 0.2)


def test_reference_arm_only_rank0_prints(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    class A:  # noqa: E701
        workload, seed, steps, warmup = "cluster24", 0, 1, 0
    assert bench.run_reference(A, rank=1, world=2) is None

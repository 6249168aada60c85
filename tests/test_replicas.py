"""Multi-GPU runs are replicas (each rank its own index and query batch, no
collective on the data path); the one cross-rank step is the whole-job
throughput: all ranks' queries over the slowest rank's time.  Checked with
two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, elapsed = bench.job_throughput(1.0 + rank, 1000.0)
    q.put((rank, value, elapsed))
    dist.destroy_process_group()


def test_job_throughput_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # 2 ranks x 1000 queries over the slower rank's 2 s
    assert got == [(0, 1000.0, 2.0), (1, 1000.0, 2.0)]


def test_single_process_is_its_own_job():
    import bench
    assert bench.job_throughput(0.5, 1000.0) == (2000.0, 0.5)

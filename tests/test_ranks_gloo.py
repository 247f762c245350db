"""The benchmark's multi-GPU path shards one video by frame range (weak scaling, no
collective on the data path): each rank times its own frames, rank 0 reports the slowest
rank's time and the whole job's pixels over it. The rank logic runs here as two gloo
processes on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)  # rank 1 is the slower one
    rate = bench.job_rate(1000 * 800 * 600, world, ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, rate))


def test_two_ranks_report_the_slowest_rank_and_the_whole_job():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in res:
        assert ms == 15.0
        assert rate == pytest.approx(2 * 1000 * 800 * 600 / 0.015 / 1e6)

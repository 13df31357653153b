"""Host logic of bench.py for N replicas (one process per GPU, no data-path collective):
whole-job rate = all ranks' units / the slowest rank's time.  Run as two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    rate, ms = bench.whole_job_rate(160, 100.0 + 50.0 * rank, dist, "cpu")   # rank 1 is slower
    q.put((rank, rate, ms))
    dist.destroy_process_group()


def test_whole_job_rate_uses_slowest_rank_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, ms in res:
        assert ms == pytest.approx(150.0)
        assert rate == pytest.approx(2 * 160 / 0.150)


def test_whole_job_rate_single_process():
    import bench
    rate, ms = bench.whole_job_rate(32, 20.0)
    assert (rate, ms) == (pytest.approx(1600.0), 20.0)

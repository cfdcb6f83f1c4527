"""World-size-2 gloo run of the multi-rank aggregation bench.py uses (no GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2401_16732_gb300.dist import max_over_ranks, whole_job_rate
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [2.0, 5.0][rank]  # rank 1 is slower
        rate, slowest = whole_job_rate(units_per_rank=20.0, seconds_this_rank=secs)
        q.put((rank, rate, slowest, max_over_ranks(float(rank + 10))))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_two_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, rate, slowest, mx in got:
        assert slowest == 5.0  # the slowest rank's time
        assert rate == pytest.approx(2 * 20.0 / 5.0)  # all ranks' units over it
        assert mx == 11.0


def test_single_process_is_identity():
    from paper_2401_16732_gb300.dist import max_over_ranks, whole_job_rate
    assert max_over_ranks(3.5) == 3.5
    assert whole_job_rate(10.0, 2.0) == (5.0, 2.0)

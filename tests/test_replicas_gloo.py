"""The multi-rank path of the benchmark on CPU: two gloo ranks, each with its
own replica's timing and work counter, aggregate to the slowest rank's time
and the summed work (weak scaling, no collective on the data path)."""
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


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.rank_env()
        ms = 10.0 + 5.0 * r          # rank 1 is the slow one
        units = 1000.0 * (r + 1)
        value, ms_max, total = bench.whole_job_rate(units, ms, w)
        out.put((r, w, lr, value, ms_max, total, bench.reduce_over_ranks(r, "sum", w)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, w, lr, value, ms_max, total, rsum) in enumerate(res):
        assert (rank, w, lr) == (r, 2, r)
        assert ms_max == 15.0 and total == 3000.0 and rsum == 1.0
        assert value == pytest.approx(3000.0 / 0.015)


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(500.0, 2.0, 1) == (250000.0, 2.0, 500.0)

"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): pages are
sharded by rank (distinct seeds, no collective on the data path), the step
time is the max over ranks, and the whole-job rate counts every rank's units."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                     # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms)
    rate = bench.whole_job_rate(100, world, ms_max)
    r, w, lr = bench.env_rank()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms_max, rate, r, w))


def test_two_ranks_max_time_and_whole_job_rate():
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
    for rank, ms_max, rate, r, w in res:
        assert ms_max == pytest.approx(15.0)
        assert rate == pytest.approx(100 * 2 / 0.015)
        assert (r, w) == (rank, 2)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(10, 1, 2.0) == pytest.approx(5000.0)


def test_ranks_get_distinct_pages():
    import bench
    a = bench.make_pages(1, seed_base=0)[0]
    b = bench.make_pages(1, seed_base=160)[0]
    assert a.shape == b.shape and (a != b).any()

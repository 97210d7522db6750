"""The multi-GPU path is replicas: every rank runs its own batch (or its own
serving requests) with no exchange of data, and the reported rate is the units
of all ranks over the slowest rank's time.  These world-size-2 tests run the
host side of that path on CPU with the gloo backend."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, rk, local = bench._dist()
        my_ms = 10.0 + 5.0 * rank                         # rank 1 is the slow one
        ms = bench.max_over_ranks(my_ms, dist, "cpu")
        rate = bench.whole_job_rate(1000, ws, ms)
        ids = [r["id"] for r in bench.rank_requests(6, rk)]
        dist.barrier()
        out.put((rank, ws, rk, local, ms, rate, ids))
    finally:
        dist.destroy_process_group()


def test_replicas_world_size_2():
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
    (r0, ws0, rk0, l0, ms0, rate0, ids0), (r1, ws1, rk1, l1, ms1, rate1, ids1) = res
    assert (ws0, ws1, rk0, rk1, l0, l1) == (2, 2, 0, 1, 0, 1)
    assert ms0 == ms1 == 15.0                              # every rank reports the slowest rank's time
    assert rate0 == rate1 == pytest.approx(2 * 1000 / 0.015)
    assert ids0 == list(range(0, 6)) and ids1 == list(range(6, 12))   # disjoint requests per rank


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.whole_job_rate(500, 1, 1000.0) == 500.0

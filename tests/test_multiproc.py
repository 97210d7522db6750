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


# ---- one transform across processes (the digit cut of Algorithm 1) ----------
# Each gloo rank holds one block of the samples, runs the stages of its low
# digits, takes part in one all-to-all, and runs the stages of the top digits;
# the ranks' results, placed at their coefficient labels, must be the oracle's
# transform of the whole function, and the inverse must give the blocks back.
# The digit stages here are numpy's FFT along the digit axes of the block (the
# p-point DFT of Sec. 2.2 along chosen digits); on the GPU they are the
# library's dwt_forward_digits (tests/test_gpu_shard.py).

def _np_stages(p, m_local):
    import numpy as np
    import torch

    def st(inp, out, d0, nd, sgn):
        a = inp.numpy().astype(np.complex128) if not inp.is_complex() else inp.numpy()
        arr = a.reshape([p] * m_local)                 # axis k holds digit m_local - 1 - k
        axes = [m_local - 1 - d for d in range(d0, d0 + nd)]
        r = np.fft.fftn(arr, axes=axes) / p ** nd if sgn < 0 else np.fft.ifftn(arr, axes=axes) * p ** nd
        r = r.reshape(-1)
        out.copy_(torch.from_numpy(r.real.copy() if not out.is_complex() else r))

    return st


def _shard_worker(rank, world, port, p, m, g, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import numpy as np
    import torch
    import torch.distributed as dist

    import synthetic as S
    from paper_0808_0487_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        N = p ** m
        f = S.uniform(S.stream_seed(40, S.P_VALUES, p * 100 + m), N) - 0.5
        lo, hi = shard.block_of(rank, p, m, g)
        cplx = p > 2
        dt = torch.complex128 if cplx else torch.float64
        x = torch.from_numpy(f[lo:hi].astype(np.complex128) if cplx else f[lo:hi].copy())
        T = shard.ShardedTransform(p, m, g, _np_stages(p, m - g), shard.torch_exchange())
        work = torch.empty(hi - lo, dtype=dt)
        res = torch.empty(hi - lo, dtype=dt)
        T.forward(x, work, res)
        coef = res.numpy().copy()
        back = torch.empty(hi - lo, dtype=dt)
        T.inverse(res.clone(), work, back)
        out.put((rank, coef, shard.coefficient_index(rank, p, m, g), back.numpy().copy(), f[lo:hi]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("p,m,g,world", [(2, 10, 1, 2), (3, 4, 1, 3), (2, 6, 2, 4)])
def test_sharded_transform_gloo(orc, p, m, g, world):
    import numpy as np

    import synthetic as S
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, p, m, g, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    N = p ** m
    f = S.uniform(S.stream_seed(40, S.P_VALUES, p * 100 + m), N) - 0.5
    ref = orc.fwt(p, m, f)
    seen = np.zeros(N, dtype=bool)
    for rank, coef, H, back, fblk in got:
        H = np.asarray(H)
        assert np.abs(coef - ref[H]).max() < 1e-12
        seen[H] = True
        assert np.abs(back - fblk).max() < 1e-12
    assert seen.all()                                   # every coefficient lives on exactly one rank

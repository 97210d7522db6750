"""The digit-range stages (dwt_forward_digits / dwt_inverse_digits) and the
transform split across processes (paper_0808_0487_gb300.shard) on one GPU.

Sec. 2.2: the transform is the Kronecker product of one p-point DFT per digit,
so the stages of a partition of the digits compose, in any order, to the whole
transform.  Checked against the oracle's Algorithm 1 and against dwt_forward.
The sharded transform runs its G processes one after another in this one
process (their steps do not wait on each other inside any kernel): every
block's low stages, then the all-to-all as copies of the pieces between the
blocks, then every block's top stages; the results, placed at their
coefficient labels, must be the oracle's transform of the whole function."""
import numpy as np
import pytest
import torch

import synthetic as S
from conftest import rel_l2
from paper_0808_0487_gb300 import shard

pytestmark = pytest.mark.gpu


def _data(p, m, idx):
    N = p ** m
    return S.uniform(S.stream_seed(41, S.P_VALUES, 1000 * p + 10 * m + idx), N) - 0.5


@pytest.mark.parametrize("p,m,cuts", [(2, 12, [5, 9]), (2, 20, [7]), (3, 9, [2, 6]), (5, 6, [3]), (17, 3, [1, 2])])
def test_digit_ranges_compose_to_the_transform(dwt, dev, orc, p, m, cuts):
    N = p ** m
    f = _data(p, m, 0)
    plan = dwt.dwt_plan_create(p, m, 1, S.small_net(p, m, 1, index=5), dwt.DWT_PLAN_TRANSFORM_ONLY)
    edges = [0] + cuts + [m]
    ranges = [(edges[i], edges[i + 1] - edges[i]) for i in range(len(edges) - 1)]
    ref = orc.fwt(p, m, f)
    if p == 2:
        x = torch.tensor(f.astype(np.float32), device=dev)
        y = x.clone()
        for d0, nd in reversed(ranges):                  # top digits first: any order composes
            dwt.dwt_forward_digits(plan, y, y, 1, N, N, dwt.DWT_F32, dwt.DWT_F32, d0, nd)
        got = y.double().cpu().numpy()
        assert rel_l2(got, ref.real) < 1e-5
        full = torch.empty_like(x)
        dwt.dwt_forward(plan, x, full, 1, N, N, dwt.DWT_F32, dwt.DWT_F32)
        assert rel_l2(got, full.double().cpu().numpy()) < 1e-5
        for d0, nd in ranges:
            dwt.dwt_inverse_digits(plan, y, y, 1, N, N, dwt.DWT_F32, dwt.DWT_F32, d0, nd)
        assert rel_l2(y.double().cpu().numpy(), f) < 1e-5
    else:
        x = torch.tensor(f.astype(np.float32), device=dev)
        y = torch.empty(N, dtype=torch.complex64, device=dev)
        d0, nd = ranges[0]
        dwt.dwt_forward_digits(plan, x, y, 1, N, N, dwt.DWT_F32, dwt.DWT_C64, d0, nd)   # real in, first range
        for d0, nd in ranges[1:]:
            dwt.dwt_forward_digits(plan, y, y, 1, N, N, dwt.DWT_C64, dwt.DWT_C64, d0, nd)
        got = y.cpu().numpy().astype(np.complex128)
        assert rel_l2(got, ref) < 1e-5
        for d0, nd in reversed(ranges):
            dwt.dwt_inverse_digits(plan, y, y, 1, N, N, dwt.DWT_C64, dwt.DWT_C64, d0, nd)
        assert rel_l2(y.cpu().numpy().astype(np.complex128), f) < 1e-5


def test_digit_ranges_int32_bit_exact(dwt, dev, orc):
    p, m = 2, 16
    N = p ** m
    v = S.int_values(S.stream_seed(41, S.P_INTS, 1), 1, N)[0]
    plan = dwt.dwt_plan_create(p, m, 1, S.small_net(p, m, 1, index=6), dwt.DWT_PLAN_TRANSFORM_ONLY)
    x = torch.tensor(v, device=dev)
    for d0, nd in [(11, 5), (0, 6), (6, 5)]:
        dwt.dwt_forward_digits(plan, x, x, 1, N, N, dwt.DWT_I32, dwt.DWT_I32, d0, nd)
    assert np.array_equal(x.cpu().numpy().astype(np.int64), orc.fwt_i64(m, v.astype(np.int64)))


def test_digit_ranges_reject_bad_ranges(dwt, dev):
    plan = dwt.dwt_plan_create(2, 8, 1, S.small_net(2, 8, 1), dwt.DWT_PLAN_TRANSFORM_ONLY)
    x = torch.zeros(256, device=dev)
    for d0, nd in [(-1, 2), (0, 0), (5, 4), (8, 1)]:
        with pytest.raises(dwt.DwtError) as e:
            dwt.dwt_forward_digits(plan, x, x, 1, 256, 256, dwt.DWT_F32, dwt.DWT_F32, d0, nd)
        assert e.value.status == dwt.DWT_EINVAL


@pytest.mark.parametrize("p,m,g", [(2, 16, 1), (2, 18, 3), (3, 8, 2), (5, 5, 1), (2, 10, 0)])
def test_sharded_transform_on_one_gpu(dwt, dev, orc, p, m, g):
    N = p ** m
    G = p ** g
    L = N // G
    f = _data(p, m, 1)
    T = shard.ShardedTransform(p, m, g, shard.LibraryStages(p, m - g), exchange=None)
    cplx = p > 2
    dt = torch.complex64 if cplx else torch.float32
    x = [torch.tensor(f[slice(*shard.block_of(r, p, m, g))].astype(np.float32), device=dev) for r in range(G)]
    work = [torch.empty(L, dtype=dt, device=dev) for _ in range(G)]
    res = [torch.empty(L, dtype=dt, device=dev) for _ in range(G)]
    if g == 0:
        T.forward(x[0], work[0], res[0])
    else:
        for r in range(G):
            T.low(x[r], work[r])
        chunk = L // G                                   # the all-to-all: piece r' of block r -> block r', at r
        for r in range(G):
            for rr in range(G):
                res[rr][r * chunk:(r + 1) * chunk] = work[r][rr * chunk:(rr + 1) * chunk]
        for r in range(G):
            T.top(res[r])
    ref = orc.fwt(p, m, f)
    got = np.empty(N, dtype=np.complex128)
    for r in range(G):
        got[np.asarray(shard.coefficient_index(r, p, m, g))] = res[r].cpu().numpy()
    assert rel_l2(got if cplx else got.real, ref if cplx else ref.real) < 1e-5
    # and back
    back = [torch.empty(L, dtype=dt, device=dev) for _ in range(G)]
    if g == 0:
        T.inverse(res[0], work[0], back[0])
    else:
        for r in range(G):
            T.top_inverse(res[r], work[r])
        for r in range(G):
            for rr in range(G):
                back[rr][r * chunk:(r + 1) * chunk] = work[r][rr * chunk:(rr + 1) * chunk]
        for r in range(G):
            T.low_inverse(back[r])
    bh = np.concatenate([b.cpu().numpy() for b in back])
    assert rel_l2(bh if cplx else bh.real, f) < 1e-5

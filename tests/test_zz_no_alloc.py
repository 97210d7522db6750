"""dwt_effdim_static, the allocation-free effective-dimension call, against
dwt_effdim_packed.

Some callers cannot let the library allocate device memory (a fixed memory
budget owned by the host program, or a loop that cannot take the device-wide
synchronisation of cudaMalloc / cudaFree).  dwt_effdim_static keeps its
scratch in a fixed array inside the library instead.  This test calls it
through the C ABI twice in a row on a fresh plan, before any other call has
given the plan a workspace, checks with the library's allocation counter that
those calls allocated nothing, then checks both results against
dwt_effdim_packed within the tolerance of the other variance tests (relative
1e-5, dimensions exact).  One case is large enough (p = 2, m = 24, s = 32,
batch 9: 135,234 partials per function, 7 functions per pass through the
array) that the batch goes through the array in two groups.  An over-size
request is refused with a message that names the limit.
The file is named so that pytest collects it last."""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _case(dwt, dev, p, m, s, B, idx):
    if p == 2 and m == 20:
        C = S.workload_p2_m20()["C"]
    elif p == 2 and m == 24:
        C = S.workload_p2_m24(batch=1)["C"]
    else:
        C = S.small_net(p, m, s, index=idx)
    plan = dwt.dwt_plan_create(p, m, s, C)
    N = p ** m
    g = S.uniform(S.stream_seed(30, S.P_VALUES, idx), B * (2 if p != 2 else 1) * N) - 0.5
    if p == 2:
        coef = torch.tensor(g.reshape(B, N).astype(np.float32), device=dev)
        t = dwt.DWT_F32
    else:
        coef = torch.tensor(g.reshape(B, 2 * N).astype(np.float32), device=dev)
        t = dwt.DWT_C64
    return plan, coef, t, N


@pytest.mark.parametrize("p,m,s,B", [(2, 20, 16, 12), (3, 8, 5, 3), (2, 12, 4, 2), (2, 24, 32, 9)])
def test_effdim_static_matches_effdim(dwt, dev, p, m, s, B):
    plan, coef, t, N = _case(dwt, dev, p, m, s, B, idx=m)
    torch.cuda.synchronize()
    got = []
    a0 = dwt.dwt_alloc_count()
    for _ in range(2):                              # two calls in a row share the array
        var = torch.full((B, 2, s + 1), -1.0, dtype=torch.float64, device=dev)
        dim = torch.full((B, 2), -1, dtype=torch.int32, device=dev)
        a1 = dwt.dwt_alloc_count()
        dwt.dwt_effdim_static(plan, coef, B, N, t, var=var, dim=dim, threshold=0.95)
        torch.cuda.synchronize()
        assert dwt.dwt_alloc_count() == a1          # the call itself allocated nothing
        got.append((var.cpu().numpy(), dim.cpu().numpy()))
    assert dwt.dwt_alloc_count() == a0
    var_ref = torch.empty((B, 2, s + 1), dtype=torch.float64, device=dev)
    dim_ref = torch.empty((B, 2), dtype=torch.int32, device=dev)
    dwt.dwt_effdim_packed(plan, coef, B, N, t, var=var_ref, dim=dim_ref, threshold=0.95)
    torch.cuda.synchronize()
    assert dwt.dwt_alloc_count() > a0               # the ordinary call grew the plan's workspace
    vr, dr = var_ref.cpu().numpy(), dim_ref.cpu().numpy()
    for v, d in got:
        assert np.allclose(v, vr, rtol=1e-5, atol=0.0)
        assert np.array_equal(d, dr)


def test_effdim_static_rejects_oversize(dwt, dev):
    # 2 (s+1) (ceil(N/8192) + 1) partials per function must fit 2^20 doubles:
    # s = 255 at N = 2^24 needs 2 * 256 * 2049 > 2^20 and is refused before any work
    p, m, s = 2, 24, 255
    C = np.stack([np.eye(m, dtype=np.uint8)] * s)
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    x = torch.zeros(2 ** m, device=dev)
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt_effdim_static(plan, x, 1, 2 ** m, dwt.DWT_F32)
    assert e.value.status == dwt.DWT_EINVAL
    assert "scratch" in str(e.value) and "1048576" in str(e.value)
    # s = 40 at N = 2^20 needs 2 * 41 * 129 and is served
    plan2 = dwt.dwt_plan_create(2, 20, 40, S.small_net(2, 20, 40, index=1))
    big = torch.zeros(2 ** 20, device=dev)
    dim = torch.full((1, 2), -1, dtype=torch.int32, device=dev)
    dwt.dwt_effdim_static(plan2, big, 1, 2 ** 20, dwt.DWT_F32, dim=dim)
    assert dim.cpu().numpy().tolist() == [[0, 0]]          # zero variance -> d = 0

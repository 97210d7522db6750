"""dwt_effdim_static, the allocation-free effective-dimension call, against dwt_effdim.

Some callers cannot let the library allocate device memory (a fixed memory
budget owned by the host program, or a loop that cannot take the device-wide
synchronisation of cudaMalloc / cudaFree).  dwt_effdim_static keeps its
scratch in a fixed array inside the library instead.  This test calls it
through the C ABI twice in a row on the same inputs and checks both results
against dwt_effdim within the tolerance of the other variance tests
(relative 1e-5, dimensions exact), and that an over-size request is refused.
The file is named so that pytest collects it last."""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _case(dwt, dev, p, m, s, B, idx):
    C = S.small_net(p, m, s, index=idx) if p != 2 or m != 20 else S.workload_p2_m20()["C"]
    plan = dwt.dwt_plan_create(p, m, s, C)
    N = p ** m
    g = S.uniform(S.stream_seed(30, S.P_VALUES, idx), B * 2 * N) - 0.5
    if p == 2:
        coef = torch.tensor(g[:B * N].reshape(B, N).astype(np.float32), device=dev)
        t = dwt.DWT_F32
    else:
        coef = torch.tensor(g.reshape(B, 2 * N).astype(np.float32), device=dev)
        t = dwt.DWT_C64
    return plan, coef, t, N


@pytest.mark.parametrize("p,m,s,B", [(2, 20, 16, 12), (3, 8, 5, 3), (2, 12, 4, 2)])
def test_effdim_static_matches_effdim(dwt, dev, p, m, s, B):
    plan, coef, t, N = _case(dwt, dev, p, m, s, B, idx=m)
    var_ref = torch.empty((B, 2, s + 1), dtype=torch.float64, device=dev)
    dim_ref = torch.empty((B, 2), dtype=torch.int32, device=dev)
    dwt.dwt_effdim(plan, coef, B, N, t, var=var_ref, dim=dim_ref, threshold=0.95)
    for _ in range(2):                              # two calls in a row share the array
        var = torch.full((B, 2, s + 1), -1.0, dtype=torch.float64, device=dev)
        dim = torch.full((B, 2), -1, dtype=torch.int32, device=dev)
        dwt.dwt_effdim_static(plan, coef, B, N, t, var=var, dim=dim, threshold=0.95)
        torch.cuda.synchronize()
        assert np.allclose(var.cpu().numpy(), var_ref.cpu().numpy(), rtol=1e-5, atol=0.0)
        assert np.array_equal(dim.cpu().numpy(), dim_ref.cpu().numpy())


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
    # s = 40 at N = 2^20 needs 2 * 41 * 129 and is served
    plan2 = dwt.dwt_plan_create(2, 20, 40, S.small_net(2, 20, 40, index=1))
    big = torch.zeros(2 ** 20, device=dev)
    dim = torch.full((1, 2), -1, dtype=torch.int32, device=dev)
    dwt.dwt_effdim_static(plan2, big, 1, 2 ** 20, dwt.DWT_F32, dim=dim)
    assert dim.cpu().numpy().tolist() == [[0, 0]]          # zero variance -> d = 0

"""The split-BF16 tensor-core form of the p = 2 transform (DWT_ALGO_TC_SPLIT_BF16):
relative L2 error against the FP64 oracle <= 1e-5, forward and inverse."""
import numpy as np
import pytest
import torch

import synthetic as S
from conftest import rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m", [14, 18, 20, 24])
def test_tc_forward_inverse(dwt, dev, orc, m):
    p, N, B = 2, 2 ** m, 2
    C = S.small_net(p, m, 2, index=m + 50)
    plan = dwt.dwt_plan_create(p, m, 2, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    v = S.uniform(S.stream_seed(31, S.P_VALUES, m), B * N) - 0.5
    f = v.reshape(B, N)
    fin = torch.tensor(f.astype(np.float32), device=dev)
    out = torch.empty_like(fin)
    dwt.dwt_forward(plan, fin, out, B, N, N, dwt.DWT_F32, dwt.DWT_F32, dwt.DWT_ALGO_TC_SPLIT_BF16)
    got = out.cpu().numpy()
    for b in range(B):
        assert rel_l2(got[b], orc.fwt(p, m, f[b]).real) < 1e-5
    back = torch.empty_like(fin)
    dwt.dwt_inverse(plan, out, back, B, N, N, dwt.DWT_F32, dwt.DWT_F32, dwt.DWT_ALGO_TC_SPLIT_BF16)
    assert rel_l2(back.cpu().numpy(), f) < 1e-5


def test_tc_product_function_m24(dwt, dev, orc):
    """The bench's function family on a p = 2, m = 24 net."""
    w = S.workload_p2_m24(batch=1)
    p, m, s = w["p"], w["m"], w["s"]
    N = p ** m
    plan = dwt.dwt_plan_create(p, m, s, w["C"], dwt.DWT_PLAN_TRANSFORM_ONLY)
    coef = torch.tensor(w["coef"], device=dev)
    f = torch.empty((1, N), device=dev)
    dwt.dwt_eval_product(plan, coef, f, 1, N, dwt.DWT_F32)
    ref = torch.empty_like(f)
    dwt.dwt_forward(plan, f, ref, 1, N, N, dwt.DWT_F32, dwt.DWT_F32)
    tc = torch.empty_like(f)
    dwt.dwt_forward(plan, f, tc, 1, N, N, dwt.DWT_F32, dwt.DWT_F32, dwt.DWT_ALGO_TC_SPLIT_BF16)
    f64 = f.double().cpu().numpy()[0]
    exact = orc.fwt(p, m, f64).real
    assert rel_l2(tc.cpu().numpy()[0], exact) < 1e-5
    assert rel_l2(ref.cpu().numpy()[0], exact) < 1e-5

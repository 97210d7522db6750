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


def _check_dims(got, dt, ds, vt, vs, thr=0.99):
    tot = vt[-1]
    for d_got, d_ref, v in ((got[0], dt, vt), (got[1], ds, vs)):
        if d_got != d_ref:
            lo, hi = sorted((d_got, d_ref))
            assert all(abs(v[d] / tot - thr) < 1e-5 for d in range(lo, hi)), (d_got, d_ref)


@pytest.mark.parametrize("m,s,B", [(18, 6, 3), (20, 12, 2), (24, 8, 2)])
def test_tc_interpolate(dwt, dev, orc, m, s, B):
    """dwt_interpolate with the low passes of both transforms on the tensor cores
    (several functions: the launches that pair one function's inverse with the
    next one's forward).  The split error is relative to the norm of the data,
    so the class variances are compared relative to the total variance."""
    p, N = 2, 2 ** m
    C = S.small_net(p, m, s, index=m + 60)
    plan = dwt.dwt_plan_create(p, m, s, C)
    Y = orc.net_points(p, m, C)
    coefs = S.uniform(S.stream_seed(32, S.P_COEFFS, m), B * s).reshape(B, s)
    fs = np.stack([orc.eval_product(p, m, Y, coefs[b]) for b in range(B)])
    tab = orc.coset_leaders_dp(p, m, C)
    fin = torch.tensor(fs.astype(np.float32), device=dev)
    c = torch.empty((B, N), device=dev)
    var = torch.empty((B, 2, s + 1), dtype=torch.float64, device=dev)
    dim = torch.empty((B, 2), dtype=torch.int32, device=dev)
    dwt.dwt_interpolate(plan, fin, c, None, B, N, dwt.DWT_F32, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER,
                        dwt.DWT_ALGO_TC_SPLIT_BF16, var=var, dim=dim)
    cg, vg, dg = c.cpu().numpy(), var.cpu().numpy(), dim.cpu().numpy()
    for b in range(B):
        cref, g, vt, vs, dt, ds = orc.interpolate(p, m, fs[b], tab["W64"], tab["cls"], s)
        assert rel_l2(cg[b], cref.real) < 1e-5
        tot = vt[-1]
        assert np.all(np.abs(vg[b, 0] - vt) <= 1e-5 * tot)
        assert np.all(np.abs(vg[b, 1] - vs) <= 1e-5 * tot)
        _check_dims(dg[b], dt, ds, vt, vs)


def test_tc_interpolate_rejects_small_m(dwt, dev):
    p, m, s = 2, 16, 4
    plan = dwt.dwt_plan_create(p, m, s, S.small_net(p, m, s, index=3))
    f = torch.zeros(2 ** m, device=dev)
    c = torch.empty_like(f)
    with pytest.raises(dwt.DwtError):
        dwt.dwt_interpolate(plan, f, c, None, 1, 2 ** m, dwt.DWT_F32, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER,
                            dwt.DWT_ALGO_TC_SPLIT_BF16)


def test_bounded_wait_gives_up_and_context_survives(dwt, dev, orc):
    """A device wait that never completes returns DWT_ETIMEOUT instead of hanging,
    and the tensor-core path still works afterwards."""
    assert dwt.dwt_selftest_bounded_wait() == dwt.DWT_ETIMEOUT
    assert "bounded wait" in dwt.lib().dwt_last_error().decode()
    p, m, N = 2, 14, 2 ** 14
    plan = dwt.dwt_plan_create(p, m, 1, S.small_net(p, m, 1, index=2), dwt.DWT_PLAN_TRANSFORM_ONLY)
    v = S.uniform(S.stream_seed(33, S.P_VALUES), N) - 0.5
    x = torch.tensor(v.astype(np.float32), device=dev)
    y = torch.empty_like(x)
    dwt.dwt_forward(plan, x, y, 1, N, N, dwt.DWT_F32, dwt.DWT_F32, dwt.DWT_ALGO_TC_SPLIT_BF16)
    assert rel_l2(y.cpu().numpy(), orc.fwt(p, m, v).real) < 1e-5

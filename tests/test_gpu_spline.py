"""GPU parity of the kernel spline (Sec. 3.1) and its ANOVA variances (Sec. 4)
against the FP64 oracle.  Both sides divide f~ by p^m K~; the rounding of K~
(about 1e-16 of the largest kernel datum) is amplified where K~ is small, so
the tolerance on c is that ratio, measured on the oracle's K~."""
import numpy as np
import pytest
import torch

import synthetic as S
from conftest import rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p,m,s,alpha,B,pad", [(2, 10, 4, 2.0, 1, 0), (2, 14, 6, 2.0, 2, 4), (3, 7, 3, 2.0, 1, 0),
                                              (5, 5, 4, 2.5, 2, 3), (2, 16, 8, 1.7, 3, 0), (7, 4, 3, 2.0, 1, 1),
                                              (17, 3, 3, 2.0, 1, 1), (31, 2, 3, 2.5, 2, 0)])
def test_spline_matches_oracle(dwt, dev, orc, p, m, s, alpha, B, pad):
    N = p ** m
    ld = N + pad
    C = S.small_net(p, m, s, index=200 + m)
    Y = orc.net_points(p, m, C)
    gamma = 0.9 / np.arange(1, s + 1) ** 1.2
    coefs = S.uniform(S.stream_seed(60, S.P_COEFFS, m), B * s).reshape(B, s)
    fs = np.stack([orc.eval_product(p, m, Y, coefs[b]) for b in range(B)])
    refs = [orc.spline(p, m, Y, fs[b], alpha, gamma) for b in range(B)]
    K, _, _ = orc.kernel_data(p, m, Y, alpha, gamma)
    cond = np.abs(K).max() / np.abs(refs[0]["Ktil"].real).min()
    tol_c = max(1e-11, 1e-15 * cond * 50)

    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    dwt.dwt_spline_prepare(plan, alpha, gamma)
    f = torch.zeros((B, ld), dtype=torch.float64, device=dev)
    f[:, :N] = torch.from_numpy(fs)
    cdt = torch.float64 if p == 2 else torch.complex128
    c = torch.zeros((B, ld), dtype=cdt, device=dev)
    vt = torch.empty((B, s + 1), dtype=torch.float64, device=dev)
    vs = torch.empty((B, s + 1), dtype=torch.float64, device=dev)
    dim = torch.empty((B, 2), dtype=torch.int32, device=dev)
    dwt.dwt_spline(plan, f, c, B, ld, vt, vs, dim)
    cg = c.cpu().numpy()[:, :N]
    vtg, vsg, dg = vt.cpu().numpy(), vs.cpu().numpy(), dim.cpu().numpy()
    for b in range(B):
        r = refs[b]
        assert rel_l2(cg[b].real, r["c"].real) < tol_c
        tot = r["var_trc"][-1]
        assert np.all(np.abs(vtg[b] - r["var_trc"]) <= 1e-9 * tot)
        assert np.all(np.abs(vsg[b] - r["var_sup"]) <= 1e-9 * tot)
        for dgot, dref, v in ((dg[b, 0], r["d_trc"], r["var_trc"]), (dg[b, 1], r["d_sup"], r["var_sup"])):
            if dgot != dref:
                lo, hi = sorted((dgot, dref))
                assert all(abs(v[d] / tot - 0.99) < 1e-8 for d in range(lo, hi))


def test_spline_needs_prepare(dwt, dev):
    p, m, s = 2, 8, 3
    plan = dwt.dwt_plan_create(p, m, s, S.small_net(p, m, s, index=1), dwt.DWT_PLAN_TRANSFORM_ONLY)
    f = torch.zeros(2 ** m, dtype=torch.float64, device=dev)
    with pytest.raises(dwt.DwtError):
        dwt.dwt_spline(plan, f, f.clone(), 1, 2 ** m)
    with pytest.raises(dwt.DwtError):
        dwt.dwt_spline_prepare(plan, 1.0, np.ones(s))   # alpha must exceed 1


@pytest.mark.parametrize("p,m,s,M,B", [(2, 10, 4, 11, 2), (2, 14, 5, 15, 1), (3, 6, 3, 7, 1), (5, 4, 3, 6, 2),
                                       (2, 12, 3, 12, 1)])
def test_spline_values_shifted(dwt, dev, orc, p, m, s, M, B):
    """Values at x_n (+) delta and the hold-out squared error, against the oracle's DWT
    route (itself pinned by the direct kernel sum)."""
    N = p ** m
    C = S.small_net(p, m, s, index=210 + m)
    Y = orc.net_points(p, m, C)
    gamma = 0.8 / np.arange(1, s + 1)
    alpha = 2.0
    coefs = S.uniform(S.stream_seed(62, S.P_COEFFS, m), B * s).reshape(B, s)
    fs = np.stack([orc.eval_product(p, m, Y, coefs[b]) for b in range(B)])
    delta = S.integers(S.stream_seed(63, S.P_SAMPLE, m), s, 0, p ** M - 1).astype(np.uint32)
    K, _, _ = orc.kernel_data(p, m, Y, alpha, gamma)
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    dwt.dwt_spline_prepare(plan, alpha, gamma)
    cdt = torch.float64 if p == 2 else torch.complex128
    f = torch.from_numpy(fs).to(dev)
    c = torch.empty((B, N), dtype=cdt, device=dev)
    dwt.dwt_spline(plan, f, c, B, N)
    vals = torch.empty_like(c)
    fshift = torch.from_numpy(fs[::-1].copy()).to(dev)   # any data at the shifted points
    sse = torch.empty(B, dtype=torch.float64, device=dev)
    dwt.dwt_spline_values_shifted(plan, c, delta, M, vals, B, N, fshift, sse)
    vg = vals.cpu().numpy()
    ref0 = orc.spline(p, m, Y, fs[0], alpha, gamma)
    tol = max(1e-10, 1e-15 * 50 * np.abs(K).max() / np.abs(ref0["Ktil"].real).min())
    for b in range(B):
        cref = orc.spline(p, m, Y, fs[b], alpha, gamma)["c"].real
        ref = orc.spline_values_shifted(p, m, Y, cref, delta, M, alpha, gamma).real
        assert rel_l2(vg[b].real, ref) < tol
        err = float(((fs[::-1][b] - ref) ** 2).sum())
        assert sse.cpu().numpy()[b] == pytest.approx(err, rel=max(1e-8, 10 * tol), abs=1e-14)


# (2, 8, 40, 20, 9, 130): s > 32 (narrower net tiles), two function blocks and
# two point blocks; (2, 12, 3, 12, 1, 129): M = m (no digits below the net's)
@pytest.mark.parametrize("p,m,s,M,B,Q", [(2, 10, 4, 14, 2, 300), (2, 12, 3, 12, 1, 129), (3, 6, 3, 9, 1, 200),
                                         (5, 4, 3, 6, 2, 150), (7, 4, 2, 5, 1, 64), (13, 3, 2, 4, 1, 50),
                                         (2, 8, 40, 20, 9, 130), (3, 5, 2, 20, 3, 257), (17, 3, 2, 5, 1, 70),
                                         (31, 2, 3, 6, 2, 40)])
def test_spline_eval_matches_oracle(dwt, dev, orc, p, m, s, M, B, Q):
    """Sf at arbitrary points against the oracle's direct sum, both from the
    oracle's coefficients (so only the evaluation is compared)."""
    N = p ** m
    ld = N + 3
    C = S.small_net(p, m, s, index=230 + m)
    Y = orc.net_points(p, m, C)
    gamma = 0.8 / np.arange(1, s + 1) ** 1.3
    alpha = 1.8
    coefs = S.uniform(S.stream_seed(64, S.P_COEFFS, m), B * s).reshape(B, s)
    cs = np.stack([orc.spline(p, m, Y, orc.eval_product(p, m, Y, coefs[b]), alpha, gamma)["c"] for b in range(B)])
    X = S.integers(S.stream_seed(65, S.P_SAMPLE, m), Q * s, 0, p ** M - 1).astype(np.uint32).reshape(Q, s)
    X[0] = (Y[:, N // 2].astype(np.uint64) * p ** (M - m)).astype(np.uint32)   # a net point itself
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    dwt.dwt_spline_prepare(plan, alpha, gamma)
    cdt = torch.float64 if p == 2 else torch.complex128
    c = torch.zeros((B, ld), dtype=cdt, device=dev)
    c[:, :N] = torch.from_numpy(cs if p != 2 else cs.real.copy())
    Xd = torch.from_numpy(X.view(np.int32)).to(dev)
    vals = torch.full((B, Q + 5), np.nan, dtype=torch.float64, device=dev)
    dwt.dwt_spline_eval(plan, c, B, ld, Xd, Q, M, vals, Q + 5)
    vg = vals.cpu().numpy()
    kmax = np.prod(1.0 + gamma)
    for b in range(B):
        ref = orc.spline_eval(p, m, Y, cs[b].real, X, M, alpha, gamma)
        scale = np.abs(cs[b].real).sum() * kmax
        assert np.allclose(vg[b, :Q], ref, rtol=1e-12, atol=1e-13 * scale)
        assert np.all(np.isnan(vg[b, Q:]))


def test_spline_eval_full_size_sampled(dwt, dev, orc):
    """p = 2, m = 20, s = 16, a batch of 32 and 256 points (the timed launch
    shape): eight points checked against the oracle's direct sum."""
    w = S.workload_p2_m20()
    p, m, s, C = w["p"], w["m"], 16, w["C"][:16]
    N, B, Q, M = 2 ** m, 32, 256, 24
    Y = orc.net_points(p, m, C)
    gamma = 0.9 / np.arange(1, s + 1) ** 1.2
    alpha = 2.0
    f = orc.eval_product(p, m, Y, w["coef"][0][:s])
    c0 = orc.spline(p, m, Y, f, alpha, gamma)["c"].real
    X = S.integers(S.stream_seed(66, S.P_SAMPLE, 0), Q * s, 0, 2 ** 24 - 1).astype(np.uint32).reshape(Q, s)
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    dwt.dwt_spline_prepare(plan, alpha, gamma)
    c = torch.from_numpy(c0).to(dev).unsqueeze(0).repeat(B, 1).contiguous()
    vals = torch.empty((B, Q), dtype=torch.float64, device=dev)
    dwt.dwt_spline_eval(plan, c, B, N, torch.from_numpy(X.view(np.int32)).to(dev), Q, M, vals)
    vg = vals.cpu().numpy()
    pick = S.sample_indices(8, Q, index=3)
    ref = orc.spline_eval(p, m, Y, c0, X[pick], M, alpha, gamma)
    scale = np.abs(c0).sum() * np.prod(1.0 + gamma)
    for b in (0, 13, 31):
        assert np.allclose(vg[b, pick], ref, rtol=1e-12, atol=1e-13 * scale)


def test_spline_eval_rejects_bad_calls(dwt, dev):
    p, m, s = 3, 4, 2
    N = p ** m
    plan = dwt.dwt_plan_create(p, m, s, S.small_net(p, m, s, index=2), dwt.DWT_PLAN_TRANSFORM_ONLY)
    c = torch.zeros(N, dtype=torch.complex128, device=dev)
    X = torch.zeros((4, s), dtype=torch.int32, device=dev)
    v = torch.empty(4, dtype=torch.float64, device=dev)
    with pytest.raises(dwt.DwtError):           # no dwt_spline_prepare yet
        dwt.dwt_spline_eval(plan, c, 1, N, X, 4, 6, v)
    dwt.dwt_spline_prepare(plan, 2.0, np.ones(s))
    with pytest.raises(dwt.DwtError):           # M < m
        dwt.dwt_spline_eval(plan, c, 1, N, X, 4, m - 1, v)
    with pytest.raises(dwt.DwtError):           # 3^21 > 2^32
        dwt.dwt_spline_eval(plan, c, 1, N, X, 4, 21, v)
    dwt.dwt_spline_eval(plan, c, 1, N, X, 0, 6, v)   # no points: nothing to do
    dwt.dwt_spline_eval(plan, c, 1, N, X, 4, 6, v)
    assert np.all(v.cpu().numpy() == 0.0)        # zero coefficients

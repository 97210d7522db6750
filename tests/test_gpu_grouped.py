"""Grouped transforms (dwt_forward_grouped / dwt_inverse_grouped): the calls of
several plans with nets of different sizes in few launches.  Every output
element must be bit-identical to the job's own dwt_forward / dwt_inverse call
(Algorithm 1 / Algorithm 2 per job), and one job is also checked against the
oracle's transform."""
import numpy as np
import pytest
import torch

import synthetic as S
from conftest import rel_l2

pytestmark = pytest.mark.gpu


def _plan(dwt, p, m, idx):
    return dwt.dwt_plan_create(p, m, 1, S.small_net(p, m, 1, index=idx), dwt.DWT_PLAN_TRANSFORM_ONLY)


def _real(p, m, batch, idx, ld=None):
    N = p ** m
    ld = ld or N
    x = np.zeros((batch, ld), dtype=np.float64)
    x[:, :N] = (S.uniform(S.stream_seed(43, S.P_VALUES, 100 * p + 10 * m + idx), batch * N) - 0.5).reshape(batch, N)
    return x


def _same_bits(a, b):
    return torch.equal(a.contiguous().view(torch.int32), b.contiguous().view(torch.int32))


# p = 2: generic passes (m <= 11, 15), the one-tile low pass (12 .. 14), and
# the register-tile pair (m >= 16, own launches); one strided job, one in place
P2_JOBS = [(5, 3), (9, 1), (11, 2), (12, 4), (13, 1), (14, 2), (15, 3), (17, 1), (12, 2), (7, 5)]


@pytest.mark.parametrize("dtype", ["f32", "i32"])
def test_grouped_p2_bit_identical(dwt, dev, dtype, orc):
    tt = torch.float32 if dtype == "f32" else torch.int32
    dt = dwt.DWT_F32 if dtype == "f32" else dwt.DWT_I32
    jobs, ref_in, outs, plans = [], [], [], []
    for i, (m, b) in enumerate(P2_JOBS):
        N = 2 ** m
        ld = N + 4 if i == 1 else N                        # one job with ld > N
        plan = _plan(dwt, 2, m, i)
        x = _real(2, m, b, i, ld)
        if dtype == "i32":
            x = np.rint(x * 1000)
        xin = torch.tensor(x, dtype=tt, device=dev)
        out = xin if i == 2 else torch.zeros_like(xin)     # one job in place
        ref = torch.zeros_like(xin)
        dwt.dwt_forward(plan, xin.clone(), ref, b, ld, ld, dt, dt)
        plans.append(plan)
        ref_in.append((xin.clone(), ld, b))
        outs.append((out, ref))
        jobs.append((plan, xin, out, b, ld, ld))
    dwt.dwt_profile_reset()
    dwt.dwt_profile_enable(True)
    dwt.dwt_forward_grouped(jobs, dt, dt)
    torch.cuda.synchronize()
    dwt.dwt_profile_enable(False)
    n_lo = dwt.dwt_profile_query("grouped_lo")[0]
    n_gp = dwt.dwt_profile_query("grouped_pass")[0]
    dwt.dwt_profile_reset()
    assert n_lo == 3                                       # sizes 2^12, 2^13, 2^14: one launch each
    assert n_gp == max(len(dwt.dwt_plan_passes(pl, 4)) for pl, (m, _) in zip(plans, P2_JOBS) if m < 12 or m == 15)
    for i, ((out, ref), (m, b)) in enumerate(zip(outs, P2_JOBS)):
        N = 2 ** m
        assert _same_bits(out[:, :N], ref[:, :N]), "job %d (m = %d)" % (i, m)
    # the inverse, grouped, back to the inputs (and bit-identical to the own calls)
    back = [torch.zeros_like(o) for o, _ in outs]
    dwt.dwt_inverse_grouped([(pl, ref, bk, b, ld, ld) for pl, (_, ref), bk, (_, ld, b) in
                             zip(plans, outs, back, ref_in)], dt, dt)
    for (pl, (_, ref), bk, (xin, ld, b), (m, _)) in zip(plans, outs, back, ref_in, P2_JOBS):
        own = torch.zeros_like(bk)
        dwt.dwt_inverse(pl, ref, own, b, ld, ld, dt, dt)
        N = 2 ** m
        assert _same_bits(bk[:, :N], own[:, :N])
        if dtype == "i32":   # D (G f) = N f exactly
            assert torch.equal(bk[:, :N], xin[:, :N] * N)
    # one job against the oracle
    m, b = P2_JOBS[3]
    if dtype == "f32":
        f = ref_in[3][0][0].double().cpu().numpy()
        assert rel_l2(outs[3][0][0].double().cpu().numpy(), orc.fwt(2, m, f).real) < 1e-5


@pytest.mark.parametrize("p,ms,cplx_in", [(3, [3, 5, 7, 9, 4], False), (5, [2, 4, 6, 3], True), (7, [2, 3, 5], False),
                                          (31, [2, 3], True)])
def test_grouped_odd_bit_identical(dwt, dev, orc, p, ms, cplx_in):
    jobs, checks = [], []
    for i, m in enumerate(ms):
        N = p ** m
        b = 1 + i % 3
        plan = _plan(dwt, p, m, i)
        x = _real(p, m, b, i)
        if cplx_in:
            xin = torch.tensor(x + 0.25j * x[:, ::-1], dtype=torch.complex64, device=dev)
            it = dwt.DWT_C64
        else:
            xin = torch.tensor(x, dtype=torch.float32, device=dev)
            it = dwt.DWT_F32
        out = torch.zeros((b, N), dtype=torch.complex64, device=dev)
        ref = torch.zeros_like(out)
        dwt.dwt_forward(plan, xin, ref, b, N, N, it, dwt.DWT_C64)
        jobs.append((plan, xin, out, b, N, N))
        checks.append((plan, xin, out, ref, b, N, m))
    dwt.dwt_forward_grouped(jobs, it, dwt.DWT_C64)
    for plan, xin, out, ref, b, N, m in checks:
        assert _same_bits(torch.view_as_real(out), torch.view_as_real(ref)), "p %d m %d" % (p, m)
    plan, xin, out, ref, b, N, m = checks[-1]
    f = xin[0].cpu().numpy().astype(np.complex128)
    assert rel_l2(out[0].cpu().numpy().astype(np.complex128), orc.fwt(p, m, f)) < 1e-5
    # inverse, grouped and in place, bit-identical to the own calls
    mine = [(c[2].clone(), c) for c in checks]
    dwt.dwt_inverse_grouped([(c[0], x, x, c[4], c[5], c[5]) for x, c in mine], dwt.DWT_C64, dwt.DWT_C64)
    for x, (plan, xin, out, ref, b, N, m) in mine:
        own = torch.zeros_like(out)
        dwt.dwt_inverse(plan, out, own, b, N, N, dwt.DWT_C64, dwt.DWT_C64)
        assert _same_bits(torch.view_as_real(x), torch.view_as_real(own))


def test_grouped_f64(dwt, dev):
    jobs, checks = [], []
    for i, m in enumerate([4, 6, 8]):
        N = 3 ** m
        plan = _plan(dwt, 3, m, i)
        xin = torch.tensor(_real(3, m, 2, i), dtype=torch.float64, device=dev)
        out = torch.zeros((2, N), dtype=torch.complex128, device=dev)
        ref = torch.zeros_like(out)
        dwt.dwt_forward(plan, xin, ref, 2, N, N, dwt.DWT_F64, dwt.DWT_C128)
        jobs.append((plan, xin, out, 2, N, N))
        checks.append((out, ref))
    dwt.dwt_forward_grouped(jobs, dwt.DWT_F64, dwt.DWT_C128)
    for out, ref in checks:
        assert torch.equal(torch.view_as_real(out), torch.view_as_real(ref))


def test_grouped_rejects_bad_lists(dwt, dev):
    p2 = _plan(dwt, 2, 6, 0)
    p3 = _plan(dwt, 3, 4, 0)
    x = torch.zeros(81, dtype=torch.complex64, device=dev)
    y = torch.zeros(64, device=dev)
    for jobs, it, ot in (([], dwt.DWT_F32, dwt.DWT_F32),
                         ([(p2, y, y, 1, 64, 64), (p3, x, x, 1, 81, 81)], dwt.DWT_F32, dwt.DWT_F32),
                         ([(p2, y, y, 1, 32, 64)], dwt.DWT_F32, dwt.DWT_F32),
                         ([(p2, y, y, 1, 64, 64)], dwt.DWT_F32, dwt.DWT_C64)):
        with pytest.raises(dwt.DwtError) as e:
            dwt.dwt_forward_grouped(jobs, it, ot)
        assert e.value.status in (dwt.DWT_EINVAL, dwt.DWT_EUNSUPPORTED)
    # batch 0 jobs are skipped
    dwt.dwt_forward_grouped([(p2, None, None, 0, 64, 64)], dwt.DWT_F32, dwt.DWT_F32)

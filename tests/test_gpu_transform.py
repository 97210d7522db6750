"""GPU parity of Algorithms 1 and 2 (dwt_forward / dwt_inverse) against the oracle.

Tolerances: relative L2 per function <= 1e-5 for FP32 / complex FP32 and
<= 1e-12 for FP64; the int32 p = 2 path is bit-exact."""
import numpy as np
import pytest
import torch

import synthetic as S
from conftest import rel_l2

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12


def _np(t):
    return t.detach().cpu().numpy()


def _cplx(t):
    a = _np(t)
    return a[..., 0::2] + 1j * a[..., 1::2]


def test_pr1_f64_vs_direct_sum(dwt, dev, orc):
    w = S.workload_pr1()
    p, m, s, C = w["p"], w["m"], w["s"], w["C"]
    N = p ** m
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    f = orc.eval_product(p, m, orc.net_points(p, m, C), w["coef"][0])
    ref = orc.dwt_direct(p, m, f).real
    fin = torch.tensor(f, device=dev)
    out = torch.empty(N, dtype=torch.float64, device=dev)
    dwt.dwt_forward(plan, fin, out, 1, N, N, dwt.DWT_F64, dwt.DWT_F64)
    assert rel_l2(_np(out), ref) < TOL64
    back = torch.empty_like(out)
    dwt.dwt_inverse(plan, out, back, 1, N, N, dwt.DWT_F64, dwt.DWT_F64)
    assert rel_l2(_np(back), f) < TOL64
    # FP32 path on the same input
    f32 = torch.tensor(f.astype(np.float32), device=dev)
    o32 = torch.empty(N, device=dev)
    dwt.dwt_forward(plan, f32, o32, 1, N, N, dwt.DWT_F32, dwt.DWT_F32)
    assert rel_l2(_np(o32), ref) < TOL32


@pytest.mark.parametrize("pad,inplace", [(0, False), (64, False), (0, True)])
def test_p2_m20_batch_f32(dwt, dev, orc, pad, inplace):
    w = S.workload_p2_m20()
    p, m, s, C = w["p"], w["m"], w["s"], w["C"]
    N = p ** m
    B = 8 if pad or inplace else 32
    ld = N + pad
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    Y = orc.net_points(p, m, C)
    fs = np.stack([orc.eval_product(p, m, Y, w["coef"][b]) for b in range(B)])
    host = np.zeros((B, ld), dtype=np.float32)
    host[:, :N] = fs
    fin = torch.tensor(host, device=dev)
    out = fin if inplace else torch.full((B, ld), 7.0, device=dev)
    dwt.dwt_forward(plan, fin, out, B, ld, ld, dwt.DWT_F32, dwt.DWT_F32)
    got = _np(out)
    for b in range(B):
        assert rel_l2(got[b, :N], orc.fwt(p, m, fs[b]).real) < TOL32
    if pad and not inplace:
        assert (got[:, N:] == 7.0).all()          # padding untouched
    back = torch.empty((B, ld), device=dev)
    dwt.dwt_inverse(plan, out, back, B, ld, ld, dwt.DWT_F32, dwt.DWT_F32)
    gb = _np(back)
    for b in range(B):
        assert rel_l2(gb[b, :N], fs[b]) < TOL32


def test_p2_m20_int32_exact(dwt, dev, orc):
    w = S.workload_p2_m20()
    p, m, s, C = w["p"], w["m"], w["s"], w["C"]
    N = p ** m
    B = w["batch_i32"]
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    v = S.int_values(w["int_seed"], B, N)
    vin = torch.tensor(v, device=dev)
    out = torch.empty_like(vin)
    dwt.dwt_forward(plan, vin, out, B, N, N, dwt.DWT_I32, dwt.DWT_I32)
    got = _np(out)
    for b in range(0, B, 5):
        assert np.array_equal(got[b].astype(np.int64), orc.fwt_i64(m, v[b]))
    back = torch.empty_like(vin)
    dwt.dwt_inverse(plan, out, back, B, N, N, dwt.DWT_I32, dwt.DWT_I32)
    assert np.array_equal(_np(back).astype(np.int64), N * v.astype(np.int64))


def test_p3_m13_complex(dwt, dev, orc):
    w = S.workload_p3_m13()
    p, m, s, C = w["p"], w["m"], w["s"], w["C"]
    N = p ** m
    ld = (N + 3) // 4 * 4
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    f = orc.eval_exp(p, m, orc.net_points(p, m, C))
    host = np.zeros(ld, dtype=np.float32)
    host[:N] = f
    fin = torch.tensor(host, device=dev)
    out = torch.empty(2 * ld, device=dev)
    dwt.dwt_forward(plan, fin, out, 1, ld, ld, dwt.DWT_F32, dwt.DWT_C64)
    ref = orc.fwt(p, m, f)
    got = _cplx(out)[:N]
    assert rel_l2(got, ref) < TOL32
    back = torch.empty(2 * ld, device=dev)
    dwt.dwt_inverse(plan, out, back, 1, ld, ld, dwt.DWT_C64, dwt.DWT_C64)
    gb = _cplx(back)[:N]
    assert rel_l2(gb, f) < TOL32
    assert np.abs(gb.imag).max() < 1e-5 * np.abs(f).max()


# the inverse on its own (Algorithm 2 / Lemma 3.1), fed with given coefficients,
# against the oracle's FP64 Algorithm 2 of the same (FP32-rounded) coefficients,
# function by function; p = 2 at the register-tile sizes (m = 20 in a batch of
# 3 with a padded ld, m = 24 in a batch of 2) and p = 3, m = 13 (complex)
@pytest.mark.parametrize("p,m,B,pad", [(2, 20, 3, 4), (2, 24, 2, 0), (3, 13, 2, 1)])
def test_inverse_alone_vs_oracle(dwt, dev, orc, p, m, B, pad):
    N = p ** m
    ld = N + pad
    plan = dwt.dwt_plan_create(p, m, 1, S.small_net(p, m, 1, index=7), dwt.DWT_PLAN_TRANSFORM_ONLY)
    if p == 2:
        g = (S.uniform(S.stream_seed(25, S.P_VALUES, m), B * ld) - 0.5).astype(np.float32).reshape(B, ld)
        x = torch.tensor(g, device=dev)
        y = torch.full_like(x, 7.0)
        dwt.dwt_inverse(plan, x, y, B, ld, ld, dwt.DWT_F32, dwt.DWT_F32)
        yh = _np(y)
        for b in range(B):
            ref = orc.fiwt(p, m, g[b, :N].astype(np.float64)).real
            assert rel_l2(yh[b, :N], ref) < TOL32, b
            assert np.all(yh[b, N:] == 7.0)          # the padding of ld is not written
    else:
        g = (S.uniform(S.stream_seed(25, S.P_VALUES, m), 2 * B * ld) - 0.5).astype(np.float32).reshape(B, 2 * ld)
        x = torch.tensor(g, device=dev)
        y = torch.empty_like(x)
        dwt.dwt_inverse(plan, x, y, B, ld, ld, dwt.DWT_C64, dwt.DWT_C64)
        yh = _cplx(y)
        for b in range(B):
            cin = g[b, 0:2 * N:2].astype(np.float64) + 1j * g[b, 1:2 * N:2].astype(np.float64)
            ref = orc.fiwt(p, m, cin)
            assert rel_l2(yh[b, :N], ref) < TOL32, b


# sizes chosen so that the pass decomposition has 1, 2 and 3 passes and ragged tiles
@pytest.mark.parametrize("p,m", [(2, 1), (2, 14), (2, 15), (2, 25), (3, 1), (3, 9), (5, 3), (5, 10), (7, 2), (7, 8),
                                 (11, 1), (11, 5), (13, 2), (13, 5), (17, 1), (17, 4), (19, 3), (23, 2), (23, 5),
                                 (29, 3), (31, 1), (31, 4), (31, 5)])
def test_sizes_and_primes(dwt, dev, orc, p, m):
    N = p ** m
    s = 2
    C = S.small_net(p, m, s, index=m)
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    v = S.uniform(S.stream_seed(20, S.P_VALUES, p * 100 + m), 2 * N) - 0.5
    if p == 2:
        f = v[:N]
        fin = torch.tensor(f.astype(np.float32), device=dev)
        out = torch.empty(N, device=dev)
        dwt.dwt_forward(plan, fin, out, 1, N, N, dwt.DWT_F32, dwt.DWT_F32)
        assert rel_l2(_np(out), orc.fwt(p, m, f).real) < TOL32
        back = torch.empty(N, device=dev)
        dwt.dwt_inverse(plan, out, back, 1, N, N, dwt.DWT_F32, dwt.DWT_F32)
        assert rel_l2(_np(back), f) < TOL32
    else:
        f = v[:N] + 1j * v[N:]
        inter = np.empty(2 * N, dtype=np.float32)
        inter[0::2] = f.real
        inter[1::2] = f.imag
        fin = torch.tensor(inter, device=dev)
        out = torch.empty(2 * N, device=dev)
        dwt.dwt_forward(plan, fin, out, 1, N, N, dwt.DWT_C64, dwt.DWT_C64)
        assert rel_l2(_cplx(out), orc.fwt(p, m, f)) < TOL32
        back = torch.empty(2 * N, device=dev)
        dwt.dwt_inverse(plan, out, back, 1, N, N, dwt.DWT_C64, dwt.DWT_C64)
        assert rel_l2(_cplx(back), f) < TOL32


# (3, 10), (5, 6), (7, 5): a low pass and a high pass of 16-byte elements
@pytest.mark.parametrize("p,m", [(3, 7), (5, 4), (2, 16), (3, 10), (5, 6), (7, 5)])
def test_double_precision(dwt, dev, orc, p, m):
    N = p ** m
    C = S.small_net(p, m, 2, index=1)
    plan = dwt.dwt_plan_create(p, m, 2, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    f = S.uniform(S.stream_seed(21, S.P_VALUES, p), N) - 0.5
    fin = torch.tensor(f, device=dev)
    if p == 2:
        out = torch.empty(N, dtype=torch.float64, device=dev)
        dwt.dwt_forward(plan, fin, out, 1, N, N, dwt.DWT_F64, dwt.DWT_F64)
        assert rel_l2(_np(out), orc.fwt(p, m, f).real) < TOL64
    else:
        out = torch.empty(2 * N, dtype=torch.float64, device=dev)
        dwt.dwt_forward(plan, fin, out, 1, N, N, dwt.DWT_F64, dwt.DWT_C128)
        assert rel_l2(_cplx(out), orc.fwt(p, m, f)) < TOL64
        back = torch.empty_like(out)
        dwt.dwt_inverse(plan, out, back, 1, N, N, dwt.DWT_C128, dwt.DWT_C128)
        assert rel_l2(_cplx(back), f) < TOL64


def test_edge_cases(dwt, dev):
    C = S.small_net(2, 4, 1)
    plan = dwt.dwt_plan_create(2, 4, 1, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    x = torch.zeros(16, device=dev)
    assert dwt.dwt_forward(plan, x, x, 0, 16, 16, dwt.DWT_F32, dwt.DWT_F32) == 0      # empty batch
    with pytest.raises(dwt.DwtError) as e:                                            # ld < N
        dwt.dwt_forward(plan, x, x, 1, 8, 16, dwt.DWT_F32, dwt.DWT_F32)
    assert e.value.status == dwt.DWT_EINVAL
    with pytest.raises(dwt.DwtError) as e:                                            # complex out for p = 2
        dwt.dwt_forward(plan, x, x, 1, 16, 16, dwt.DWT_F32, dwt.DWT_C64)
    assert e.value.status == dwt.DWT_EUNSUPPORTED
    # zeros stay zeros; a delta at n = 0 gives the constant 1/N
    dwt.dwt_forward(plan, x, x, 1, 16, 16, dwt.DWT_F32, dwt.DWT_F32)
    assert (x == 0).all()
    x[0] = 1.0
    dwt.dwt_forward(plan, x, x, 1, 16, 16, dwt.DWT_F32, dwt.DWT_F32)
    assert torch.allclose(x, torch.full_like(x, 1 / 16))


# the register-tile p = 2 kernels: one low pass (m <= 14) or low + high pass (16 <= m <= 24)
@pytest.mark.parametrize("m", [12, 13, 14, 16, 17, 18, 19, 20, 21, 22, 23, 24])
def test_p2_register_tile_sizes(dwt, dev, orc, m):
    p, N, B = 2, 2 ** m, 2
    C = S.small_net(p, m, 2, index=m)
    plan = dwt.dwt_plan_create(p, m, 2, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    v = S.uniform(S.stream_seed(25, S.P_VALUES, m), B * N) - 0.5
    f = v.reshape(B, N)
    fin = torch.tensor(f.astype(np.float32), device=dev)
    out = torch.empty_like(fin)
    dwt.dwt_forward(plan, fin, out, B, N, N, dwt.DWT_F32, dwt.DWT_F32)
    got = _np(out)
    for b in range(B):
        assert rel_l2(got[b], orc.fwt(p, m, f[b]).real) < TOL32
    dwt.dwt_inverse(plan, out, out, B, N, N, dwt.DWT_F32, dwt.DWT_F32)
    assert rel_l2(_np(out), f) < TOL32
    iv = S.integers(S.stream_seed(25, S.P_INTS, m), N, -1000, 1000)
    ii = torch.tensor(iv.astype(np.int32), device=dev)
    io = torch.empty_like(ii)
    dwt.dwt_forward(plan, ii, io, 1, N, N, dwt.DWT_I32, dwt.DWT_I32)
    assert np.array_equal(_np(io).astype(np.int64), orc.fwt_i64(m, iv))


def test_p2_unaligned_ld_takes_generic_path(dwt, dev, orc):
    p, m, N = 2, 20, 2 ** 20
    ld = N + 1                       # rows not 16-byte aligned
    C = S.small_net(p, m, 2, index=3)
    plan = dwt.dwt_plan_create(p, m, 2, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    f = S.uniform(S.stream_seed(26, S.P_VALUES), 2 * ld) - 0.5
    fin = torch.tensor(f.astype(np.float32), device=dev)
    out = torch.empty_like(fin)
    dwt.dwt_forward(plan, fin, out, 2, ld, ld, dwt.DWT_F32, dwt.DWT_F32)
    got = _np(out)
    for b in range(2):
        assert rel_l2(got[b * ld:b * ld + N], orc.fwt(p, m, f[b * ld:b * ld + N]).real) < TOL32


# int32 through the generic passes (m outside the register-tile range): one,
# two and three passes, exact against the oracle's int64 form; values small
# enough that N max|v| < 2^31
@pytest.mark.parametrize("m,vmax", [(11, 1000), (15, 1000), (25, 60)])
def test_p2_int32_generic_passes(dwt, dev, orc, m, vmax):
    p, N = 2, 2 ** m
    plan = dwt.dwt_plan_create(p, m, 2, S.small_net(p, m, 2, index=m), dwt.DWT_PLAN_TRANSFORM_ONLY)
    iv = S.integers(S.stream_seed(28, S.P_INTS, m), N, -vmax, vmax)
    ii = torch.tensor(iv.astype(np.int32), device=dev)
    io = torch.empty_like(ii)
    dwt.dwt_forward(plan, ii, io, 1, N, N, dwt.DWT_I32, dwt.DWT_I32)
    assert np.array_equal(_np(io).astype(np.int64), orc.fwt_i64(m, iv))
    dwt.dwt_inverse(plan, io, io, 1, N, N, dwt.DWT_I32, dwt.DWT_I32)
    assert np.array_equal(_np(io).astype(np.int64), N * iv.astype(np.int64))

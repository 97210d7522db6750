"""Parity at the benchmark's full size and launch configuration: p = 2, m = 24,
s = 32, batch 32, one dwt_interpolate call over the whole batch (as bench.py
times it), plus the forward transform at the same size.

The oracle computes the net, the input function f, the K(C) tables and the
full FP64 interpolation of f (about a minute of host time).  The batch holds 32
DIFFERENT functions derived from f: f_b(n) = a_b f(n XOR v_b) + d_b with a
distinct scale a_b, digital shift v_b and offset d_b per function.  By the
shift theorem (Sec. 2.2: wal_h of n XOR v is (-1)^{v.h} wal_h of n) and
linearity, their results follow from f's exactly: f~_b(h) = a_b (-1)^{v_b.h}
f~(h) + d_b [h = 0], the weight does not see the sign, so
c_b(n) = a_b c(n XOR v_b) + d_b, the class variances scale by a_b^2 and the
effective dimensions are those of f.  Any mix-up of functions, offsets or
shifts inside the batch (e.g. one function's inverse paired with another's
forward) shows.  Checks: weight / class tables bit-exact over all 2^24
labels; c relative L2 <= 1e-5 for every function; class variances relative
1e-5 and the effective dimensions exact; forward coefficients at sampled
labels against the O(N) direct sum (|error| <= 1e-5 ||f~_b||_2); Parseval."""
import ctypes

import numpy as np
import pytest
import torch

import synthetic as S
from conftest import rel_l2

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def full(orc):
    w = S.workload_p2_m24(batch=32)
    p, m, s = w["p"], w["m"], w["s"]
    Y = orc.net_points(p, m, w["C"])
    f = orc.eval_product(p, m, Y, w["coef"][0])
    del Y
    tab = orc.coset_leaders_dp(p, m, w["C"])
    assert tab["status"] == 0
    return w, f, tab


def _read_tables(dwt, plan, N):
    Wp, Cp = dwt.dwt_plan_tables(plan)
    W = np.empty(N, dtype=np.float32)
    cls = np.empty((N, 2), dtype=np.uint8)
    rt = ctypes.CDLL("libcudart.so")
    rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    torch.cuda.synchronize()
    assert rt.cudaMemcpy(W.ctypes.data, Wp, 4 * N, 2) == 0
    assert rt.cudaMemcpy(cls.ctypes.data, Cp, 2 * N, 2) == 0
    return W, cls


def test_fullsize_interpolate_and_forward(dwt, dev, orc, full):
    w, f, tab = full
    p, m, s, B = w["p"], w["m"], w["s"], w["batch"]
    N = p ** m
    plan = dwt.dwt_plan_create(p, m, s, w["C"])
    W, cls = _read_tables(dwt, plan, N)
    assert np.array_equal(W.view(np.uint32), tab["W32"].view(np.uint32))
    assert np.array_equal(cls, tab["cls"])
    del W, cls

    # 32 distinct functions f_b(n) = a_b f(n ^ v_b) + d_b
    a = 0.5 + S.uniform(S.stream_seed(24, S.P_VALUES, 1), B)
    d = S.uniform(S.stream_seed(24, S.P_VALUES, 2), B) - 0.5
    v = S.integers(S.stream_seed(24, S.P_VALUES, 3), B, 0, N - 1)
    v[0] = 0
    idx = np.arange(N, dtype=np.int64)
    fb = torch.empty((B, N), dtype=torch.float32, device=dev)
    for b in range(B):
        fb[b] = torch.from_numpy((a[b] * f[idx ^ v[b]] + d[b]).astype(np.float32))
    c = torch.empty_like(fb)
    var = torch.empty((B, 2, s + 1), dtype=torch.float64, device=dev)
    dim = torch.empty((B, 2), dtype=torch.int32, device=dev)
    dwt.dwt_interpolate(plan, fb, c, None, B, N, dwt.DWT_F32, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER, var=var, dim=dim)
    torch.cuda.synchronize()

    cref, g, vt, vs, dt, ds = orc.interpolate(p, m, f, tab["W64"], tab["cls"], s)
    cref = cref.real
    vh = var.cpu().numpy()
    dh = dim.cpu().numpy()
    for b in range(B):
        want = a[b] * cref[idx ^ v[b]] + d[b]
        assert rel_l2(c[b].cpu().numpy(), want) < 1e-5, b
        assert np.allclose(vh[b, 0], a[b] ** 2 * vt, rtol=1e-5, atol=1e-14 * a[b] ** 2 * vt[-1]), b
        assert np.allclose(vh[b, 1], a[b] ** 2 * vs, rtol=1e-5, atol=1e-14 * a[b] ** 2 * vt[-1]), b
        assert tuple(dh[b]) == (dt, ds), b
    del c

    # forward over the same batch
    out = torch.empty_like(fb)
    dwt.dwt_forward(plan, fb, out, B, N, N, dwt.DWT_F32, dwt.DWT_F32)
    sel = S.sample_indices(64, N, index=24)
    ref = orc.dwt_direct(p, m, f, sel).real
    sel64 = torch.tensor(sel.astype(np.int64), device=dev)
    got = out[:, sel64].cpu().numpy()
    e = (out.double() ** 2).sum(dim=1).cpu().numpy()
    pc = np.array([bin(x).count("1") for x in range(256)], dtype=np.int64)

    def parity(x):
        x = np.asarray(x, dtype=np.int64)
        return (pc[x & 255] + pc[(x >> 8) & 255] + pc[(x >> 16) & 255] + pc[(x >> 24) & 255]) & 1

    for b in range(B):
        fbb = a[b] * f[idx ^ v[b]] + d[b]
        want = a[b] * (1.0 - 2.0 * parity(sel.astype(np.int64) & v[b])) * ref + d[b] * (sel == 0)
        norm = np.sqrt(np.sum(fbb * fbb) / N)                  # ||f~_b||_2 by Parseval
        assert np.abs(got[b] - want).max() <= 1e-5 * norm, b
        assert np.isclose(e[b], np.sum(fbb * fbb) / N, rtol=1e-5), b

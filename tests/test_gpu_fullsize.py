"""Parity at the benchmark's full size and launch configuration: p = 2, m = 24,
s = 32, batch 32, one dwt_interpolate call over the whole batch (as bench.py
times it), plus the forward transform at the same size.

The oracle computes the net, the input function, the K(C) tables and the full
FP64 interpolation of one function (about a minute of host time); the GPU runs
the whole batch of 32 copies.  Checks: weight / class tables bit-exact over all
2^24 labels; forward coefficients at sampled labels against the O(N) direct sum
(|error| <= 1e-5 ||f~||_2); c relative L2 <= 1e-5 for every function; class
variances relative 1e-5 and the effective dimensions exact; Parseval."""
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

    f32 = torch.tensor(f.astype(np.float32), device=dev)
    fb = f32.unsqueeze(0).repeat(B, 1).contiguous()          # 2 GiB, the bench's input shape
    c = torch.empty_like(fb)
    var = torch.empty((B, 2, s + 1), dtype=torch.float64, device=dev)
    dim = torch.empty((B, 2), dtype=torch.int32, device=dev)
    dwt.dwt_interpolate(plan, fb, c, None, B, N, dwt.DWT_F32, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER, var=var, dim=dim)
    torch.cuda.synchronize()

    cref, g, vt, vs, dt, ds = orc.interpolate(p, m, f, tab["W64"], tab["cls"], s)
    cref = cref.real
    cg = c.cpu().numpy()
    for b in range(B):
        assert rel_l2(cg[b], cref) < 1e-5, b
    v = var.cpu().numpy()
    d = dim.cpu().numpy()
    for b in range(B):
        assert np.allclose(v[b, 0], vt, rtol=1e-5, atol=1e-14 * vt[-1])
        assert np.allclose(v[b, 1], vs, rtol=1e-5, atol=1e-14 * vt[-1])
        assert tuple(d[b]) == (dt, ds)
    del c, cg

    # forward over the same batch
    out = torch.empty_like(fb)
    dwt.dwt_forward(plan, fb, out, B, N, N, dwt.DWT_F32, dwt.DWT_F32)
    sel = S.sample_indices(64, N, index=24)
    ref = orc.dwt_direct(p, m, f, sel).real
    norm = np.sqrt(np.sum(f * f) / N)                          # ||f~||_2 by Parseval
    got = out[:, torch.tensor(sel.astype(np.int64), device=dev)].cpu().numpy()
    for b in range(B):
        assert np.abs(got[b] - ref).max() <= 1e-5 * norm
    # Parseval on the GPU result of every function
    e = (out.double() ** 2).sum(dim=1).cpu().numpy()
    assert np.allclose(e, np.sum(f * f) / N, rtol=1e-5)

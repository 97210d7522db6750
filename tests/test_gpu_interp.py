"""GPU parity of the weighting / inverse / effective-dimension path (dwt_interpolate,
dwt_effdim) and of the synthetic test functions."""
import numpy as np
import pytest
import torch

import synthetic as S
from conftest import rel_l2

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def _cplx(a):
    return a[..., 0::2] + 1j * a[..., 1::2]


def _check_dims(got, dt, ds, vt, vs, thr=0.99):
    """Dimensions must agree unless the oracle's cumulative ratio is within 1e-6 of the threshold."""
    tot = vt[-1]
    for d_got, d_ref, v in ((got[0], dt, vt), (got[1], ds, vs)):
        if d_got != d_ref:
            lo, hi = sorted((d_got, d_ref))
            assert all(abs(v[d] / tot - thr) < 1e-6 for d in range(lo, hi)), (d_got, d_ref)


@pytest.mark.parametrize("weight", [1, 0])
def test_interpolate_pr1(dwt, dev, orc, weight):
    w = S.workload_pr1()
    p, m, s, C = w["p"], w["m"], w["s"], w["C"]
    N = p ** m
    plan = dwt.dwt_plan_create(p, m, s, C)
    f = orc.eval_product(p, m, orc.net_points(p, m, C), w["coef"][0])
    tab = orc.coset_leaders_dp(p, m, C)
    Wt = tab["W64"] if weight else np.ones(N)
    cref, g, vt, vs, dt, ds = orc.interpolate(p, m, f, Wt, tab["cls"], s)
    fin = torch.tensor(f.astype(np.float32), device=dev)
    c = torch.empty(N, device=dev)
    coef = torch.empty(N, device=dev)
    var = torch.empty((1, 2, s + 1), dtype=torch.float64, device=dev)
    dim = torch.empty((1, 2), dtype=torch.int32, device=dev)
    dwt.dwt_interpolate(plan, fin, c, coef, 1, N, dwt.DWT_F32, weight, var=var, dim=dim)
    assert rel_l2(_np(c), cref.real) < 1e-5
    assert rel_l2(_np(coef), g.real) < 1e-5
    if not weight:
        assert rel_l2(_np(c), f) < 1e-5         # interpolation property: c = f
    v = _np(var)[0]
    assert np.allclose(v[0], vt, rtol=1e-5, atol=1e-14 * vt[-1])
    assert np.allclose(v[1], vs, rtol=1e-5, atol=1e-14 * vt[-1])
    _check_dims(_np(dim)[0], dt, ds, vt, vs)


def test_interpolate_m20_batch(dwt, dev, orc):
    w = S.workload_p2_m20()
    p, m, s, C = w["p"], w["m"], w["s"], w["C"]
    N = p ** m
    B = 4
    plan = dwt.dwt_plan_create(p, m, s, C)
    Y = orc.net_points(p, m, C)
    fs = np.stack([orc.eval_product(p, m, Y, w["coef"][b]) for b in range(B)])
    tab = orc.coset_leaders_dp(p, m, C)
    fin = torch.tensor(fs.astype(np.float32), device=dev)
    c = torch.empty((B, N), device=dev)
    var = torch.empty((B, 2, s + 1), dtype=torch.float64, device=dev)
    dim = torch.empty((B, 2), dtype=torch.int32, device=dev)
    dwt.dwt_interpolate(plan, fin, c, None, B, N, dwt.DWT_F32, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER, var=var, dim=dim)
    cg, vg, dg = _np(c), _np(var), _np(dim)
    for b in range(B):
        cref, g, vt, vs, dt, ds = orc.interpolate(p, m, fs[b], tab["W64"], tab["cls"], s)
        assert rel_l2(cg[b], cref.real) < 1e-5
        assert np.allclose(vg[b, 0], vt, rtol=1e-5, atol=1e-14 * vt[-1])
        assert np.allclose(vg[b, 1], vs, rtol=1e-5, atol=1e-14 * vt[-1])
        _check_dims(dg[b], dt, ds, vt, vs)


# p3_m11_s40: the top pass bins in one warp (40 coordinates: 82 classes);
# p7_m6: a top pass of two digits with seven binning warps; p5_m7: lo 5 + top 2
# p17_m4 .. p31_m3: primes above 13 (one digit per register group, the
# p-point sums in conjugate pairs)
@pytest.mark.parametrize("which", ["p3_m13", "p11_m4", "p13_m4", "p3_m11_s40", "p7_m6", "p5_m7", "p17_m4", "p19_m3",
                                   "p23_m3", "p29_m3", "p31_m3"])
def test_interpolate_p_odd(dwt, dev, orc, which):
    if which == "p3_m13":
        w = S.workload_p3_m13()
        p, m, s, C = w["p"], w["m"], w["s"], w["C"]
    else:
        p, m, s = {"p11_m4": (11, 4, 5), "p13_m4": (13, 4, 3), "p3_m11_s40": (3, 11, 40), "p7_m6": (7, 6, 5),
                   "p5_m7": (5, 7, 4), "p17_m4": (17, 4, 4), "p19_m3": (19, 3, 5), "p23_m3": (23, 3, 3),
                   "p29_m3": (29, 3, 4), "p31_m3": (31, 3, 6)}[which]
        C = S.small_net(p, m, s, index=90 + p)
    N = p ** m
    plan = dwt.dwt_plan_create(p, m, s, C)
    f = orc.eval_exp(p, m, orc.net_points(p, m, C))
    tab = orc.coset_leaders_dp(p, m, C)
    cref, g, vt, vs, dt, ds = orc.interpolate(p, m, f, tab["W64"], tab["cls"], s)
    fin = torch.tensor(f.astype(np.float32), device=dev)
    c = torch.empty(2 * N, device=dev)
    coef = torch.empty(2 * N, device=dev)
    var = torch.empty((1, 2, s + 1), dtype=torch.float64, device=dev)
    dim = torch.empty((1, 2), dtype=torch.int32, device=dev)
    dwt.dwt_interpolate(plan, fin, c, coef, 1, N, dwt.DWT_F32, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER, var=var, dim=dim)
    assert rel_l2(_cplx(_np(c)), cref) < 1e-5
    assert rel_l2(_cplx(_np(coef)), g) < 1e-5
    v = _np(var)[0]
    assert np.allclose(v[0], vt, rtol=1e-5, atol=1e-14 * vt[-1])
    assert np.allclose(v[1], vs, rtol=1e-5, atol=1e-14 * vt[-1])
    _check_dims(_np(dim)[0], dt, ds, vt, vs)


@pytest.mark.parametrize("p,m,s", [(2, 12, 4), (5, 5, 3), (7, 4, 6), (11, 3, 4), (13, 3, 3), (17, 2, 4), (31, 2, 3)])
def test_effdim_standalone(dwt, dev, orc, p, m, s):
    C = S.workload_pr1()["C"] if p == 2 else S.small_net(p, m, s, index=5)
    N = p ** m
    plan = dwt.dwt_plan_create(p, m, s, C)
    tab = orc.coset_leaders_dp(p, m, C)
    B = 3
    g = (S.uniform(S.stream_seed(23, S.P_VALUES, p), 2 * B * N) - 0.5).reshape(B, 2 * N)
    if p == 2:
        gin = torch.tensor(g[:, :N].astype(np.float32), device=dev)
        gref = gin.double().cpu().numpy()
        t = dwt.DWT_F32
    else:
        gin = torch.tensor(g.astype(np.float32), device=dev)
        gref = _cplx(gin.double().cpu().numpy())
        t = dwt.DWT_C64
    var = torch.empty((B, 2, s + 1), dtype=torch.float64, device=dev)
    dim = torch.empty((B, 2), dtype=torch.int32, device=dev)
    dwt.dwt_effdim_packed(plan, gin, B, N if p == 2 else N, t, var=var, dim=dim, threshold=0.9)
    # the same sums in the separate-array layout of dwt_effdim
    vtr = torch.full((B, s + 1), -1.0, dtype=torch.float64, device=dev)
    vsu = torch.full((B, s + 1), -1.0, dtype=torch.float64, device=dev)
    dtr = torch.full((B,), -1, dtype=torch.int32, device=dev)
    dsu = torch.full((B,), -1, dtype=torch.int32, device=dev)
    dwt.dwt_effdim(plan, gin, B, N, t, var_trc=vtr, var_sup=vsu, d_trc=dtr, d_sup=dsu, threshold=0.9)
    assert np.array_equal(_np(vtr), _np(var)[:, 0]) and np.array_equal(_np(vsu), _np(var)[:, 1])
    assert np.array_equal(_np(dtr), _np(dim)[:, 0]) and np.array_equal(_np(dsu), _np(dim)[:, 1])
    for b in range(B):
        vt, vs, dt, ds = orc.effdim(gref[b], tab["cls"], s, 0.9)
        assert np.allclose(_np(var)[b, 0], vt, rtol=1e-5)
        assert np.allclose(_np(var)[b, 1], vs, rtol=1e-5)
        _check_dims(_np(dim)[b], dt, ds, vt, vs, 0.9)


@pytest.mark.parametrize("p,m,s", [(2, 12, 4), (3, 7, 5), (2, 20, 16)])
def test_eval_functions(dwt, dev, orc, p, m, s):
    C = S.workload_p2_m20()["C"] if m == 20 else (S.workload_pr1()["C"] if p == 2 else S.small_net(p, m, s, index=6))
    N = p ** m
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    Y = orc.net_points(p, m, C)
    B = 3
    coef = S.uniform(S.stream_seed(24, S.P_COEFFS, p), B * s).reshape(B, s)
    f = torch.empty((B, N), device=dev)
    dwt.dwt_eval_product(plan, torch.tensor(coef, device=dev), f, B, N, dwt.DWT_F32)
    f64 = torch.empty((B, N), dtype=torch.float64, device=dev)
    dwt.dwt_eval_product(plan, torch.tensor(coef, device=dev), f64, B, N, dwt.DWT_F64)
    for b in range(B):
        ref = orc.eval_product(p, m, Y, coef[b])
        assert np.abs(_np(f)[b] - ref).max() < 1e-5 * np.abs(ref).max()
        assert np.abs(_np(f64)[b] - ref).max() < 1e-13 * np.abs(ref).max()
    e = torch.empty((1, N), device=dev)
    dwt.dwt_eval_exp(plan, e, 1, N, dwt.DWT_F32)
    ref = orc.eval_exp(p, m, Y)
    assert np.abs(_np(e)[0] - ref).max() < 1e-5 * np.abs(ref).max()


# (15, 5), (25, 1): the generic passes (two and three of them) with the fused
# top pass `k_mid`; (16, 120): 242 classes are too many bins for the register-
# tile top pass, so this size goes the generic way too
@pytest.mark.parametrize("m,s", [(16, 5), (18, 8), (21, 12), (24, 6), (15, 5), (25, 1), (16, 120)])
def test_interpolate_p2_register_tile_sizes(dwt, dev, orc, m, s):
    p, N = 2, 2 ** m
    C = S.small_net(p, m, s, index=m)
    plan = dwt.dwt_plan_create(p, m, s, C)
    coef = S.uniform(S.stream_seed(27, S.P_COEFFS, m), s)
    f = orc.eval_product(p, m, orc.net_points(p, m, C), coef)
    tab = orc.coset_leaders_dp(p, m, C)
    assert np.array_equal(_read_W(dwt, plan, N).view(np.uint32), tab["W32"].view(np.uint32))
    cref, g, vt, vs, dt, ds = orc.interpolate(p, m, f, tab["W64"], tab["cls"], s)
    fin = torch.tensor(f.astype(np.float32), device=dev)
    c = torch.empty(N, device=dev)
    coefo = torch.empty(N, device=dev)
    var = torch.empty((1, 2, s + 1), dtype=torch.float64, device=dev)
    dim = torch.empty((1, 2), dtype=torch.int32, device=dev)
    dwt.dwt_interpolate(plan, fin, c, coefo, 1, N, dwt.DWT_F32, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER, var=var, dim=dim)
    assert rel_l2(_np(c), cref.real) < 1e-5
    assert rel_l2(_np(coefo), g.real) < 1e-5
    v = _np(var)[0]
    assert np.allclose(v[0], vt, rtol=1e-5, atol=1e-14 * vt[-1])
    assert np.allclose(v[1], vs, rtol=1e-5, atol=1e-14 * vt[-1])
    _check_dims(_np(dim)[0], dt, ds, vt, vs)


def _read_W(dwt, plan, N):
    import ctypes
    Wp, _ = dwt.dwt_plan_tables(plan)
    W = np.empty(N, dtype=np.float32)
    rt = ctypes.CDLL("libcudart.so")
    rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    torch.cuda.synchronize()
    assert rt.cudaMemcpy(W.ctypes.data, Wp, 4 * N, 2) == 0
    return W


@pytest.mark.parametrize("p,m,s", [(3, 9, 4), (5, 6, 3)])
def test_interpolate_p_odd_unweighted(dwt, dev, orc, p, m, s):
    """Weight 1 through the generic fused pass: c returns f (the interpolation
    property of the inverse, Lemma 3.1), and the class variances are those of
    f~ itself."""
    N = p ** m
    C = S.small_net(p, m, s, index=70 + p)
    plan = dwt.dwt_plan_create(p, m, s, C)
    f = orc.eval_exp(p, m, orc.net_points(p, m, C))
    tab = orc.coset_leaders_dp(p, m, C)
    cref, g, vt, vs, dt, ds = orc.interpolate(p, m, f, np.ones(N), tab["cls"], s)
    fin = torch.tensor(f.astype(np.float32), device=dev)
    c = torch.empty(2 * N, device=dev)
    var = torch.empty((1, 2, s + 1), dtype=torch.float64, device=dev)
    dim = torch.empty((1, 2), dtype=torch.int32, device=dev)
    dwt.dwt_interpolate(plan, fin, c, None, 1, N, dwt.DWT_F32, dwt.DWT_WEIGHT_NONE, var=var, dim=dim)
    got = _cplx(_np(c))
    assert rel_l2(got.real, f) < 1e-5
    assert np.abs(got.imag).max() < 1e-5 * np.abs(f).max()
    v = _np(var)[0]
    assert np.allclose(v[0], vt, rtol=1e-5, atol=1e-14 * vt[-1])
    assert np.allclose(v[1], vs, rtol=1e-5, atol=1e-14 * vt[-1])
    _check_dims(_np(dim)[0], dt, ds, vt, vs)


@pytest.mark.parametrize("p,m,s,B", [(2, 18, 6, 3), (3, 9, 4, 2), (2, 12, 4, 2)])
def test_cuda_graph_replay_matches_calls(dwt, dev, orc, p, m, s, B):
    """dwt_interpolate and dwt_forward only enqueue work, so after one ordinary
    call (which sizes the plan's workspace) they can be captured into a CUDA
    graph; a replay gives the ordinary call's results bit for bit."""
    N = p ** m
    C = S.small_net(p, m, s, index=80 + m)
    plan = dwt.dwt_plan_create(p, m, s, C)
    Y = orc.net_points(p, m, C)
    coefs = S.uniform(S.stream_seed(29, S.P_COEFFS, m), B * s).reshape(B, s)
    fs = np.stack([orc.eval_product(p, m, Y, coefs[b]) for b in range(B)])
    f = torch.tensor(fs.astype(np.float32), device=dev)
    cl = N if p == 2 else 2 * N
    c = torch.empty((B, cl), device=dev)
    var = torch.empty((B, 2, s + 1), dtype=torch.float64, device=dev)
    dim = torch.empty((B, 2), dtype=torch.int32, device=dev)
    g_out = torch.empty((B, cl), device=dev)
    out_t = dwt.DWT_F32 if p == 2 else dwt.DWT_C64

    def calls(st):
        dwt.dwt_interpolate(plan, f, c, None, B, N, dwt.DWT_F32, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER, var=var, dim=dim,
                            stream=st)
        dwt.dwt_forward(plan, f, g_out, B, N, N, dwt.DWT_F32, out_t, stream=st)

    calls(torch.cuda.current_stream())
    torch.cuda.synchronize()
    ref = [t.clone() for t in (c, var, dim, g_out)]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        calls(torch.cuda.current_stream())
    for t in (c, var, g_out):
        t.zero_()
    dim.fill_(-1)
    graph.replay()
    torch.cuda.synchronize()
    for got, want in zip((c, var, dim, g_out), ref):
        assert torch.equal(got, want)

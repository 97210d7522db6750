"""GPU parity of the F_p index maps: net points (Def. 1.1), C . k (Sec. 2.1), and the
coset representatives K(C) with their weight / class tables -- all bit-exact."""
import itertools

import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _read_tables(dwt, plan, N):
    """Copy the plan's W and cls tables to numpy via cudaMemcpy."""
    import ctypes
    Wp, Cp = dwt.dwt_plan_tables(plan)
    W = np.empty(N, dtype=np.float32)
    cls = np.empty((N, 2), dtype=np.uint8)
    rt = ctypes.CDLL("libcudart.so")
    rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    torch.cuda.synchronize()
    assert rt.cudaMemcpy(W.ctypes.data, Wp, 4 * N, 2) == 0
    assert rt.cudaMemcpy(cls.ctypes.data, Cp, 2 * N, 2) == 0
    return W, cls


NETS = [("pr1", 2, 12, 4), ("p3", 3, 6, 4), ("p5", 5, 4, 3), ("p7", 7, 3, 3), ("p11", 11, 3, 3), ("p13", 13, 3, 2)]


def _net(name, p, m, s):
    if name == "pr1":
        return S.workload_pr1()["C"]
    return S.small_net(p, m, s, index=3)


@pytest.mark.parametrize("name,p,m,s", NETS + [("p3m13", 3, 13, 8)])
def test_points_bit_exact(dwt, dev, orc, name, p, m, s):
    C = S.workload_p3_m13()["C"] if name == "p3m13" else _net(name, p, m, s)
    N = p ** m
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    Y = torch.empty((s, N + 3), dtype=torch.int32, device=dev)
    dwt.dwt_points(plan, Y, N + 3)
    got = Y.cpu().numpy()[:, :N].view(np.uint32)
    assert np.array_equal(got, orc.net_points(p, m, C))


@pytest.mark.parametrize("name,p,m,s", NETS)
def test_k_to_h_bit_exact(dwt, dev, orc, name, p, m, s):
    C = _net(name, p, m, s)
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_TRANSFORM_ONLY)
    k = S.integers(S.stream_seed(22, S.P_SAMPLE, p), 4000 * s, 0, p ** (m + 1) - 1).astype(np.uint32).reshape(4000, s)
    H = torch.empty(4000, dtype=torch.int32, device=dev)
    dwt.dwt_wavenumber_to_index(plan, torch.tensor(k.view(np.int32), device=dev), H, 4000)
    assert np.array_equal(H.cpu().numpy().view(np.uint32), orc.k_to_h(p, m, C, k))


@pytest.mark.parametrize("name,p,m,s", NETS + [("m20", 2, 20, 16), ("p3m13", 3, 13, 8)])
def test_tables_bit_exact(dwt, dev, orc, name, p, m, s):
    if name == "m20":
        C = S.workload_p2_m20()["C"]
    elif name == "p3m13":
        C = S.workload_p3_m13()["C"]
    else:
        C = _net(name, p, m, s)
    N = p ** m
    plan = dwt.dwt_plan_create(p, m, s, C)
    assert plan.status == 0
    W, cls = _read_tables(dwt, plan, N)
    ref = orc.coset_leaders_dp(p, m, C, want_W64=False)
    assert ref["status"] == 0
    assert np.array_equal(W.view(np.uint32), ref["W32"].view(np.uint32))
    assert np.array_equal(cls, ref["cls"])


@pytest.mark.parametrize("p,m,s,idx", [(2, 3, 3, 1), (2, 4, 2, 2), (3, 2, 3, 1), (5, 1, 3, 2), (3, 3, 2, 3), (2, 2, 4, 1),
                                       (11, 1, 3, 1), (13, 1, 2, 2), (17, 1, 3, 1), (19, 1, 2, 2), (23, 1, 2, 1),
                                       (29, 1, 2, 3), (31, 1, 3, 2), (17, 2, 2, 4)])
def test_dense_nets_vs_bruteforce(dwt, dev, orc, p, m, s, idx):
    C = S.dense_matrices(p, m, s, index=idx)
    st, kmap = orc.coset_leaders_bruteforce(p, m, C)
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_KEEP_INDEX_MAP)
    assert plan.status == st
    if st:
        return
    N = p ** m
    W, cls = _read_tables(dwt, plan, N)
    W32, _, cref = orc.weight_class(kmap)
    assert np.array_equal(W.view(np.uint32), W32.view(np.uint32))
    assert np.array_equal(cls, cref)
    H = torch.arange(N, dtype=torch.int32, device=dev)
    k = torch.empty((N, s), dtype=torch.int32, device=dev)
    dwt.dwt_index_to_wavenumber(plan, H, k, N)
    assert np.array_equal(k.cpu().numpy().view(np.uint32), kmap)


def test_index_to_wavenumber_pr1(dwt, dev, orc):
    w = S.workload_pr1()
    p, m, s, C = w["p"], w["m"], w["s"], w["C"]
    N = p ** m
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_KEEP_INDEX_MAP)
    sel = S.sample_indices(500, N)
    k = torch.empty((500, s), dtype=torch.int32, device=dev)
    dwt.dwt_index_to_wavenumber(plan, torch.tensor(sel.view(np.int32), device=dev), k, 500)
    ref = orc.coset_leaders_dp(p, m, C, Hsel=sel)["ksel"]
    assert np.array_equal(k.cpu().numpy().view(np.uint32), ref)


def test_rank_deficient_plan(dwt, dev):
    C = np.stack([np.diag([1, 0]).astype(np.uint8)] * 2)
    plan = dwt.dwt_plan_create(3, 2, 2, C)
    assert plan.status == dwt.DWT_ESPAN
    x = torch.zeros(18, device=dev)
    dwt.dwt_forward(plan, x, x, 1, 9, 9, dwt.DWT_F32, dwt.DWT_C64)    # transforms still allowed
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt_interpolate(plan, x, x, None, 1, 9, dwt.DWT_C64, dwt.DWT_WEIGHT_NONE)
    assert e.value.status == dwt.DWT_ESPAN
    with pytest.raises(dwt.DwtError):
        plan2 = dwt.dwt_plan_create(2, 4, 1, S.small_net(2, 4, 1), dwt.DWT_PLAN_TRANSFORM_ONLY)
        dwt.dwt_index_to_wavenumber(plan2, x, x, 1)


# Nets with N <= 2^16 build their tables in one CTA, larger ones with one launch
# per (coordinate, digit); these sizes sit on both sides of that boundary, with
# the largest s the small path takes.
@pytest.mark.parametrize("p,m,s", [(2, 16, 64), (2, 17, 6), (3, 10, 24), (5, 7, 5), (7, 5, 40), (2, 10, 2),
                                   (17, 3, 6), (19, 4, 4), (23, 3, 5), (29, 3, 3), (31, 3, 4), (31, 4, 3)])
def test_tables_small_large_boundary(dwt, dev, orc, p, m, s):
    C = S.small_net(p, m, s, index=m + s)
    N = p ** m
    plan = dwt.dwt_plan_create(p, m, s, C, dwt.DWT_PLAN_KEEP_INDEX_MAP)
    assert plan.status == 0
    W, cls = _read_tables(dwt, plan, N)
    sel = S.sample_indices(300, N, index=m)
    ref = orc.coset_leaders_dp(p, m, C, want_W64=False, Hsel=sel)
    assert ref["status"] == 0
    assert np.array_equal(W.view(np.uint32), ref["W32"].view(np.uint32))
    assert np.array_equal(cls, ref["cls"])
    k = torch.empty((300, s), dtype=torch.int32, device=dev)
    dwt.dwt_index_to_wavenumber(plan, torch.tensor(sel.view(np.int32), device=dev), k, 300)
    assert np.array_equal(k.cpu().numpy().view(np.uint32), ref["ksel"])


# Plans without DWT_PLAN_KEEP_INDEX_MAP build K(C) with the min-tree form when
# every C_j is nonsingular; the tables must equal the oracle's bit for bit, on
# one tile, several tiles, and with a coarse tree of several levels.  A net of
# less than one tile (2^11 labels for p = 2; 3^5, 5^3, 7^2 for p = 3, 5, 7)
# runs in one CTA; larger ones in tiles (2^12; 3^8, 5^5, 7^4, or 3^5, 5^3, 7^2 when the net
# has fewer than 64 of the larger) with one cooperative launch (the trees of
# the backward sweep and the representatives k_j(U)) and one launch of the
# per-label reading.
@pytest.mark.parametrize("p,m,s", [(2, 1, 3), (2, 9, 4), (2, 13, 9), (2, 14, 3), (2, 17, 20), (3, 2, 4), (3, 8, 5),
                                   (3, 11, 9), (3, 13, 3), (5, 5, 7), (5, 9, 3), (7, 4, 6), (7, 6, 10), (2, 12, 64),
                                   (2, 14, 64), (2, 15, 33), (2, 16, 2), (2, 18, 7), (2, 20, 3), (3, 12, 40),
                                   (5, 8, 33), (7, 7, 12), (3, 14, 3), (3, 6, 20), (5, 4, 9), (7, 3, 5), (3, 9, 64),
                                   (5, 7, 33)])
def test_tables_tree_form(dwt, dev, orc, p, m, s):
    C = S.small_net(p, m, s, index=100 + m + s)
    N = p ** m
    dwt.dwt_profile_reset()
    dwt.dwt_profile_enable(True)
    plan = dwt.dwt_plan_create(p, m, s, C)
    dwt.dwt_profile_enable(False)
    n = {f: dwt.dwt_profile_query(f)[0] for f in ("tree_up", "tree_one", "tree_sweep", "tree_read")}
    dwt.dwt_profile_reset()
    assert plan.status == 0
    # which form ran
    if N <= {2: 2048, 3: 243, 5: 125, 7: 49}[p]:
        assert n == {"tree_up": 0, "tree_one": 1, "tree_sweep": 0, "tree_read": 0}
    else:
        assert n == {"tree_up": 0, "tree_one": 0, "tree_sweep": 1, "tree_read": 1}
    W, cls = _read_tables(dwt, plan, N)
    ref = orc.coset_leaders_dp(p, m, C, want_W64=False)
    assert ref["status"] == 0
    assert np.array_equal(W.view(np.uint32), ref["W32"].view(np.uint32))
    assert np.array_equal(cls, ref["cls"])


def test_tables_tree_form_dense_fallback(dwt, dev, orc):
    """A net with a singular C_j (rank of all rows still m) takes the per-digit
    programme; tables still bit-exact."""
    p, m, s = 2, 10, 3
    C = S.small_net(p, m, s, index=7).copy()
    C[1, 4, :] = C[1, 3, :]   # two equal rows: C_2 singular
    N = p ** m
    plan = dwt.dwt_plan_create(p, m, s, C)
    assert plan.status == 0
    W, cls = _read_tables(dwt, plan, N)
    ref = orc.coset_leaders_dp(p, m, C, want_W64=False)
    assert np.array_equal(W.view(np.uint32), ref["W32"].view(np.uint32))
    assert np.array_equal(cls, ref["cls"])


@pytest.mark.parametrize("p,m,s,grid", [(2, 17, 12, 1), (2, 17, 12, 3), (2, 17, 12, 5), (3, 11, 7, 2),
                                        (5, 8, 6, 7), (7, 6, 5, 3)])
def test_tables_tiled_form_any_grid(dwt, dev, orc, monkeypatch, p, m, s, grid):
    """The tiled form with fewer CTAs than tiles (each CTA loops over tiles,
    representatives read across tiles it did not build): same tables."""
    C = S.small_net(p, m, s, index=77)
    monkeypatch.setenv("DWT_TILE_GRID", str(grid))
    plan = dwt.dwt_plan_create(p, m, s, C)
    monkeypatch.delenv("DWT_TILE_GRID")
    assert plan.status == 0
    W, cls = _read_tables(dwt, plan, p ** m)
    ref = orc.coset_leaders_dp(p, m, C, want_W64=False)
    assert np.array_equal(W.view(np.uint32), ref["W32"].view(np.uint32))
    assert np.array_equal(cls, ref["cls"])

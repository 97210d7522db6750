"""Pins for the oracle's coset representatives K(C), weights and classes (Sec. 2.1)."""
import itertools

import numpy as np
import pytest

import synthetic as S


def _nu1(k, p):
    n = 0
    while k:
        k //= p
        n += 1
    return n


def _nu(kv, p):
    return sum(_nu1(int(k), p) for k in kv)


TINY = [(2, 3, 3), (2, 4, 2), (3, 2, 3), (3, 2, 2), (2, 2, 4), (5, 1, 3), (3, 3, 2), (5, 2, 2), (2, 3, 4),
        (11, 1, 3), (13, 1, 2), (7, 2, 2), (17, 1, 3), (19, 1, 2), (23, 1, 2), (29, 1, 2), (31, 1, 3), (17, 2, 2)]


@pytest.mark.parametrize("p,m,s", TINY)
@pytest.mark.parametrize("idx", [0, 1])
def test_bruteforce_matches_sorted_enumeration(orc, p, m, s, idx):
    """An independent Python enumeration: sort every k in [0,p^m)^s by (nu(k), k_1, .., k_s)
    and take the first k seen in each coset; the oracle's brute force must agree."""
    C = S.dense_matrices(p, m, s, index=idx) if idx else S.small_net(p, m, s, index=idx)
    ks = np.array(list(itertools.product(range(p ** m), repeat=s)), dtype=np.uint32)
    H = orc.k_to_h(p, m, C, ks)
    key = sorted(range(len(ks)), key=lambda t: (_nu(ks[t], p), tuple(int(x) for x in ks[t])))
    ref = {}
    for t in key:
        ref.setdefault(int(H[t]), ks[t])
    st, kmap = orc.coset_leaders_bruteforce(p, m, C)
    if len(ref) < p ** m:
        assert st == 2
        return
    assert st == 0
    for h, k in ref.items():
        assert kmap[h].tolist() == k.tolist()


@pytest.mark.parametrize("p,m,s", TINY)
@pytest.mark.parametrize("idx", [0, 1, 2, 3])
def test_dp_matches_bruteforce(orc, p, m, s, idx):
    C = S.dense_matrices(p, m, s, index=idx) if idx else S.small_net(p, m, s, index=idx)
    st, kmap = orc.coset_leaders_bruteforce(p, m, C)
    d = orc.coset_leaders_dp(p, m, C, want_kmap=True)
    assert d["status"] == st
    assert (orc.rank(p, m, C) == m) == (st == 0)
    if st:
        return
    assert np.array_equal(d["kmap"], kmap)
    assert d["numin"].tolist() == [_nu(k, p) for k in kmap]
    W32, W64, cls = orc.weight_class(kmap)
    assert np.array_equal(d["W32"].view(np.uint32), W32.view(np.uint32))
    assert np.array_equal(d["W64"], W64)
    assert np.array_equal(d["cls"], cls)


def test_hand_examples(orc):
    # s = 1, C = I: C.k is the truncation of k, so k(H) = H
    C = np.eye(3, dtype=np.uint8)[None]
    d = orc.coset_leaders_dp(2, 3, C, want_kmap=True)
    assert d["kmap"][:, 0].tolist() == list(range(8))
    # s = 2, C_1 = C_2 = I: least nu is nu(H), reached by (H, 0) and (0, H); lexicographic -> (0, H)
    C2 = np.stack([np.eye(3, dtype=np.uint8)] * 2)
    d2 = orc.coset_leaders_dp(2, 3, C2, want_kmap=True)
    assert d2["kmap"].tolist() == [[0, h] for h in range(8)]
    # rank-deficient: C_1 = C_2 = diag(1, 0) over F_3
    C3 = np.stack([np.diag([1, 0]).astype(np.uint8)] * 2)
    assert orc.coset_leaders_dp(3, 2, C3)["status"] == 2


def test_weight_class_hand_values(orc):
    W32, W64, cls = orc.weight_class([[0, 3, 0, 1], [0, 0, 0, 0], [2, 0, 0, 0]])
    assert W64.tolist() == [1 / 64, 1.0, 1 / 9]
    assert cls.tolist() == [[4, 2], [0, 0], [1, 1]]
    # FP32 weight is RN(1 / RN(P)) in IEEE single arithmetic
    assert W32[2] == np.float32(1) / np.float32(9)
    big = np.array([[2 ** 20 - 1, 2 ** 3, 6]], dtype=np.uint32)
    P = (2 ** 20) ** 2 * 81 * 49
    W32b, W64b, _ = orc.weight_class(big)
    assert W32b[0] == np.float32(1) / np.float32(float(P))
    assert W64b[0] == 1.0 / float(P)
    with pytest.raises(OverflowError):
        orc.weight_class([[2 ** 32 - 1, 2 ** 32 - 1]])


@pytest.mark.parametrize("p,m,s", [(2, 12, 4), (3, 6, 4), (5, 4, 3)])
def test_dp_invariants_medium(orc, p, m, s):
    """At sizes beyond brute force: C.k(H) = H, nu(k(H)) is the least nu, and no random
    wavenumber in the same coset is smaller in (nu, lexicographic) order."""
    C = S.small_net(p, m, s, index=2) if p != 2 else S.workload_pr1()["C"]
    d = orc.coset_leaders_dp(p, m, C, want_kmap=True)
    assert d["status"] == 0
    kmap = d["kmap"]
    N = p ** m
    assert np.array_equal(orc.k_to_h(p, m, C, kmap), np.arange(N, dtype=np.uint32))
    assert kmap[0].tolist() == [0] * s
    ks = S.integers(S.stream_seed(14, S.P_SAMPLE, p), 3000 * s, 0, N - 1).reshape(3000, s).astype(np.uint32)
    # bias towards sparse vectors, where the competition is
    mask = S.integers(S.stream_seed(15, S.P_SAMPLE, p), 3000 * s, 0, 2).reshape(3000, s) == 0
    ks[mask] = 0
    H = orc.k_to_h(p, m, C, ks)
    for k, h in zip(ks, H):
        lead = kmap[h]
        a = (_nu(k, p), tuple(int(x) for x in k))
        b = (_nu(lead, p), tuple(int(x) for x in lead))
        assert b <= a
    assert d["numin"].tolist()[:200] == [_nu(k, p) for k in kmap[:200]]


def test_dp_sampled_selection(orc):
    w = S.workload_pr1()
    d = orc.coset_leaders_dp(2, 12, w["C"], want_kmap=True, Hsel=np.array([0, 5, 4095, 77], dtype=np.uint32))
    assert np.array_equal(d["ksel"], d["kmap"][[0, 5, 4095, 77]])

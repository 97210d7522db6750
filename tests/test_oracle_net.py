"""Pins for the oracle's digital-net points and wavenumber index map (Def. 1.1, Sec. 2.1-2.2)."""
import itertools

import numpy as np
import pytest

import synthetic as S


def _digit_reverse(n, p, m):
    d = []
    for _ in range(m):
        d.append(n % p)
        n //= p
    v = 0
    for x in d:            # n_0 becomes the most significant output digit
        v = v * p + x
    return v


def test_points_hand_example_p2(orc):
    # C = [[1,1],[0,1]]: n=1 -> y=(1,0) -> x=1/2; n=2 -> y=(1,1) -> x=3/4; n=3 -> y=(0,1) -> x=1/4
    C = np.array([[[1, 1], [0, 1]]], dtype=np.uint8)
    assert orc.net_points(2, 2, C).tolist() == [[0, 2, 3, 1]]


def test_points_hand_example_p3(orc):
    # C = [[1,2],[0,1]] over F_3: n=1 -> y=(1,0) -> Y=3; n=3 -> y=(2,1) -> Y=7; n=5 -> y=(1,1) -> Y=4
    C = np.array([[[1, 2], [0, 1]]], dtype=np.uint8)
    Y = orc.net_points(3, 2, C)[0]
    assert (Y[1], Y[3], Y[5]) == (3, 7, 4)


@pytest.mark.parametrize("p,m", [(2, 8), (3, 5), (5, 3)])
def test_reversed_identity_gives_n_over_N(orc, p, m):
    C = S.reversed_identity(m)[None]
    Y = orc.net_points(p, m, C)[0]
    assert (Y == np.arange(p ** m)).all()
    x = orc.net_x(p, m, Y[None])[0]
    assert (x == np.arange(p ** m) / float(p ** m)).all()


@pytest.mark.parametrize("p,m", [(2, 9), (3, 5), (5, 3)])
def test_identity_gives_radical_inverse(orc, p, m):
    C = np.eye(m, dtype=np.uint8)[None]
    Y = orc.net_points(p, m, C)[0]
    assert Y.tolist() == [_digit_reverse(n, p, m) for n in range(p ** m)]


@pytest.mark.parametrize("p,m,s", [(2, 10, 5), (3, 6, 3), (5, 4, 3)])
def test_nonsingular_coordinates_are_permutations(orc, p, m, s):
    C = S.small_net(p, m, s, index=1)
    Y = orc.net_points(p, m, C)
    for j in range(s):
        assert np.array_equal(np.sort(Y[j]), np.arange(p ** m))


def test_k_to_h_hand_example(orc):
    # h_c = sum_j sum_i C_j[i][c] k_{j,i};  C_1 = [[1,1],[0,1]], k_1 = 1 (digit 0 only): h = row 0 = (1,1) -> H = 3
    C = np.array([[[1, 1], [0, 1]]], dtype=np.uint8)
    assert orc.k_to_h(2, 2, C, [[1]]).tolist() == [3]
    assert orc.k_to_h(2, 2, C, [[2]]).tolist() == [2]
    assert orc.k_to_h(2, 2, C, [[3]]).tolist() == [1]
    assert orc.k_to_h(2, 2, C, [[4]]).tolist() == [0]      # digit 2 is truncated


@pytest.mark.parametrize("p,m,s", [(2, 4, 3), (3, 3, 2), (5, 2, 2)])
def test_character_property(orc, p, m, s):
    """eq. (char): p^-m sum_{x in P} wal_k(x) is 1 on the dual net and 0 elsewhere."""
    C = S.dense_matrices(p, m, s, index=3)
    Y = orc.net_points(p, m, C)
    ks = np.array(list(itertools.product(range(p ** m + p), repeat=s)), dtype=np.uint32)[::7]
    H = orc.k_to_h(p, m, C, ks)
    # f = 1: f~(k) = p^-m sum conj(wal_k) = conj of the character sum
    v = orc.dwt_walsh_def(p, m, Y, np.ones(p ** m), ks)
    assert np.allclose(v, (H == 0).astype(float), atol=1e-12)
    assert (H == 0).any() and (H != 0).any()


@pytest.mark.parametrize("p,m,s", [(2, 5, 3), (3, 3, 3), (5, 2, 2)])
def test_index_map_identity(orc, p, m, s):
    """Sec. 2.2: wal_k(x_n) = omega^{n.h} with h = C.k, so the Walsh-definition DWT at k
    equals the digit-DFT form at H = C.k, for any k (digits >= m included)."""
    C = S.dense_matrices(p, m, s, index=5)
    Y = orc.net_points(p, m, C)
    rng = S.integers(S.stream_seed(12, S.P_SAMPLE), 40 * s, 0, p ** (m + 2) - 1)
    ks = rng.reshape(40, s).astype(np.uint32)
    f = S.uniform(S.stream_seed(12, S.P_VALUES), p ** m) - 0.5
    a = orc.dwt_walsh_def(p, m, Y, f, ks)
    b = orc.dwt_direct(p, m, f, orc.k_to_h(p, m, C, ks))
    assert np.abs(a - b).max() < 1e-13

"""Pins for the oracle's Algorithms 1 and 2 (Sec. 2.2, Sec. 3.3) against the O(N^2)
definition, library transforms, closed forms and exact identities."""
import itertools

import numpy as np
import pytest
import scipy.linalg

import synthetic as S


def _data(p, m, idx=0, cplx=False):
    N = p ** m
    v = S.uniform(S.stream_seed(13, S.P_VALUES, idx), 2 * N) - 0.5
    return v[:N] + 1j * v[N:] if cplx else v[:N]


@pytest.mark.parametrize("p,m", [(2, 9), (3, 5), (5, 3), (2, 1), (3, 1), (11, 2), (13, 2), (11, 1), (17, 2), (19, 1),
                                 (23, 2), (29, 1), (31, 2)])
def test_fwt_matches_direct_sum(orc, p, m):
    f = _data(p, m, cplx=p > 2)
    a = orc.fwt(p, m, f)
    b = orc.dwt_direct(p, m, f)
    assert np.abs(a - b).max() < 1e-13


@pytest.mark.parametrize("m", [1, 4, 10])
def test_p2_is_sylvester_hadamard(orc, m):
    """s = 1, C = J, p = 2: the textbook Walsh-Hadamard transform in natural order."""
    N = 2 ** m
    f = _data(2, m, 1)
    ref = scipy.linalg.hadamard(N) @ f / N
    assert np.abs(orc.fwt(2, m, f) - ref).max() < 1e-14


@pytest.mark.parametrize("p,m", [(3, 6), (5, 4), (3, 2), (11, 3), (13, 2), (17, 3), (19, 2), (23, 2), (29, 2),
                                 (31, 3)])
def test_p_odd_is_multidimensional_dft(orc, p, m):
    """F_p^{(x)m} with omega^{-nh}: numpy's forward FFT over an m-axis p x ... x p array."""
    f = _data(p, m, 2, cplx=True)
    ref = np.fft.fftn(f.reshape([p] * m)).reshape(-1) / p ** m
    assert np.abs(orc.fwt(p, m, f) - ref).max() < 1e-14


@pytest.mark.parametrize("p,m", [(2, 12), (3, 7), (5, 5), (11, 3), (13, 3), (17, 3), (31, 3)])
def test_inverse_is_identity_and_lemma(orc, p, m):
    """Lemma 3.1 / Alg. 2: c_n = sum_H c~(H) omega^{n.h}; forward then inverse is the identity."""
    f = _data(p, m, 3, cplx=p > 2)
    back = orc.fiwt(p, m, orc.fwt(p, m, f))
    assert np.linalg.norm(back - f) / np.linalg.norm(f) < 1e-13
    ct = _data(p, min(m, 5), 4, cplx=True)
    mm = min(m, 5)
    # inverse direct sum via the forward one: sum_H c(H) w^{+n.h} = N conj(DWT(conj c))
    ref = p ** mm * np.conj(orc.dwt_direct(p, mm, np.conj(ct)))
    # N-term FP64 sums: the bound scales with the size of the result
    assert np.abs(orc.fiwt(p, mm, ct) - ref).max() < 1e-13 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("p,m", [(2, 11), (3, 6), (5, 4)])
def test_parseval_and_linearity(orc, p, m):
    f = _data(p, m, 5, cplx=p > 2)
    g = _data(p, m, 6, cplx=p > 2)
    F = orc.fwt(p, m, f)
    assert abs(np.sum(np.abs(F) ** 2) - np.sum(np.abs(f) ** 2) / p ** m) < 1e-13 * np.sum(np.abs(f) ** 2)
    a, b = 0.75, -1.25
    assert np.abs(orc.fwt(p, m, a * f + b * g) - (a * F + b * orc.fwt(p, m, g))).max() < 1e-14


@pytest.mark.parametrize("p,m", [(2, 8), (3, 5), (5, 3), (19, 2), (29, 2)])
def test_shift_theorem(orc, p, m):
    """g_n = f_{n (+) v}  ->  g~(H) = omega^{v.h} f~(H)."""
    N = p ** m
    f = _data(p, m, 7, cplx=True)
    v = 5 % N
    nd = np.array([[(n // p ** r) % p for r in range(m)] for n in range(N)])
    vd = nd[v]
    idx = ((nd + vd) % p) @ (p ** np.arange(m))
    G = orc.fwt(p, m, f[idx])
    F = orc.fwt(p, m, f)
    ph = np.exp(2j * np.pi * ((nd @ vd) % p) / p)      # rows of nd double as digit vectors of H
    assert np.abs(G - ph * F).max() < 1e-14


@pytest.mark.parametrize("m", [1, 6, 14])
def test_integer_path_exact(orc, m):
    N = 2 ** m
    v = S.integers(S.stream_seed(13, S.P_INTS, m), N, -1000, 1000)
    G = orc.fwt_i64(m, v)
    ref = np.rint(orc.fwt(2, m, v.astype(float)).real * N).astype(np.int64)
    assert np.array_equal(G, ref)
    assert np.array_equal(orc.fiwt_i64(m, G), N * v)
    if m <= 10:
        assert np.array_equal(G, scipy.linalg.hadamard(N).astype(np.int64) @ v)


def test_product_function_closed_form_pr1(orc):
    """On a p = 2 net, 1 + c(x - 1/2) = (1 - c 2^{-m-1}) - sum_i c 2^{-i-1} wal_{2^{i-1}}(x)
    exactly (x has m binary digits), so f = prod_j(...) is a finite Walsh series and
    its discrete coefficients are the aliasing sums of eq. (aliasing): f~(H) = sum_{C.k = H} f^(k)."""
    w = S.workload_pr1()
    p, m, s, C, c = w["p"], w["m"], w["s"], w["C"], w["coef"][0]
    Y = orc.net_points(p, m, C)
    f = orc.eval_product(p, m, Y, c)
    F = orc.fwt(p, m, f)
    # univariate coefficients on k in {0, 2^{i-1}}
    ks1 = [0] + [2 ** (i - 1) for i in range(1, m + 1)]
    coefs = []
    for j in range(s):
        coefs.append([1 - c[j] * 2.0 ** (-m - 1)] + [-c[j] * 2.0 ** (-i - 1) for i in range(1, m + 1)])
    combos = np.array(list(itertools.product(range(m + 1), repeat=s)))
    kv = np.array(ks1, dtype=np.uint32)[combos]
    val = np.ones(len(combos))
    for j in range(s):
        val *= np.array(coefs[j])[combos[:, j]]
    H = orc.k_to_h(p, m, C, kv)
    ref = np.zeros(p ** m)
    np.add.at(ref, H, val)
    assert np.abs(F.real - ref).max() < 1e-13
    assert np.abs(F.imag).max() == 0.0
    # and the O(N^2) direct sum agrees on the same net
    assert np.abs(orc.dwt_direct(p, m, f) - F).max() < 1e-13


def test_exp_function_closed_form_p3(orc):
    """p = 3: exp(x/j^2) = prod_i phi_i(x_i) with phi_i(v) = exp(v 3^{-i}/j^2); each digit factor
    expands in characters omega^{kappa x_i} = wal_{kappa 3^{i-1}}(x), giving f^ in closed form."""
    p, m, s = 3, 3, 2
    C = S.small_net(p, m, s, index=7)
    Y = orc.net_points(p, m, C)
    f = orc.eval_exp(p, m, Y)
    w = np.exp(2j * np.pi / p)
    uni = []
    for j in range(s):
        fj = np.ones(p ** m, dtype=complex)
        for k in range(p ** m):
            for i in range(1, m + 1):
                kap = (k // p ** (i - 1)) % p
                fj[k] *= sum(np.exp(v * p ** (-i) / (j + 1) ** 2) * w ** (-kap * v) for v in range(p)) / p
        uni.append(fj)
    ks = np.array(list(itertools.product(range(p ** m), repeat=s)), dtype=np.uint32)
    val = uni[0][ks[:, 0]] * uni[1][ks[:, 1]]
    H = orc.k_to_h(p, m, C, ks)
    ref = np.zeros(p ** m, dtype=complex)
    np.add.at(ref, H, val)
    assert np.abs(orc.fwt(p, m, f) - ref).max() < 1e-13

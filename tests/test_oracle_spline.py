"""Pins of the oracle's kernel spline (Sec. 3.1) and its ANOVA variances (Sec. 4),
each against something other than the FWT route it uses:

- the short forms of K'(x, 0) and R'(x, 0) against their Walsh series with the
  printed coefficients (for x with m digits and x != 0 only k < p^m contribute:
  the terms with top digit a >= m sum a full character sum over the low digits,
  which vanishes);
- the spline coefficients against a dense solve of the interpolation
  conditions f(x_n) = sum_v c_v K(x_n (-) x_v, 0) (Sec. 3.1);
- the truncation / superposition variances against the double sums
  sigma^2((Sf)_u) = gamma_u^2 sum_{n,v} c_n c_v R_u(x_{n,u} (-) x_{v,u}, 0) of Sec. 4
  over every nonempty u."""
import itertools

import numpy as np
import pytest

import synthetic as S


def _digits(v, p, m):
    return [(v // p ** i) % p for i in range(m)]


def _khat(p, alpha, k):
    a = int(np.floor(np.log(k) / np.log(p) + 1e-12)) if k > 0 else -1
    while p ** (a + 1) <= k:
        a += 1
    while a > 0 and p ** a > k:
        a -= 1
    return (p ** alpha - p) / (p ** alpha * (p - 1)) * p ** (-alpha * a)


def _wal1(p, m, k, Y):
    # x = Y / p^m, x_i = digit m - i of Y (i = 1..m); wal_k(x) = omega^{sum_i k_{i-1} x_i}
    e = sum(((k // p ** (i - 1)) % p) * ((Y // p ** (m - i)) % p) for i in range(1, m + 1)) % p
    return np.exp(2j * np.pi * e / p)


@pytest.mark.parametrize("p,m,alpha", [(2, 5, 2.0), (2, 4, 1.5), (3, 3, 2.0), (5, 2, 3.0), (17, 1, 2.0), (19, 2, 2.5)])
def test_short_forms_equal_walsh_series(orc, p, m, alpha):
    N = p ** m
    for Y in range(1, N):
        kser = sum(_khat(p, alpha, k) * _wal1(p, m, k, Y) for k in range(1, N))
        rser = sum(_khat(p, alpha, k) ** 2 * _wal1(p, m, k, Y) for k in range(1, N))
        assert abs(kser.imag) < 1e-12 and abs(rser.imag) < 1e-12
        assert orc.kprime(p, m, alpha, Y) == pytest.approx(kser.real, abs=1e-12)
        assert orc.rprime(p, m, alpha, Y) == pytest.approx(rser.real, abs=1e-12)
    # x = 0: the full series, sum_k khat = 1 and sum_k khat^2 in closed form
    C = (p ** alpha - p) / (p ** alpha * (p - 1))
    assert orc.kprime(p, m, alpha, 0) == 1.0
    assert orc.rprime(p, m, alpha, 0) == pytest.approx(C * C * (p - 1) / (1 - p ** (1 - 2 * alpha)), rel=1e-13)


def _dsub(a, b, p, m):
    return sum((((a // p ** i) - (b // p ** i)) % p) * p ** i for i in range(m))


def _kernel_matrix(orc, p, m, Y, alpha, gamma, fn):
    s, N = Y.shape
    M = np.ones((N, N))
    for n in range(N):
        for v in range(N):
            for j in range(s):
                M[n, v] *= 1.0 + gamma[j] * fn(p, m, alpha, _dsub(int(Y[j, n]), int(Y[j, v]), p, m))
    return M


@pytest.mark.parametrize("p,m,s,alpha", [(2, 6, 3, 2.0), (3, 4, 2, 2.0), (2, 5, 4, 1.7), (5, 3, 2, 2.5)])
def test_spline_coefficients_solve_interpolation(orc, p, m, s, alpha):
    C = S.small_net(p, m, s, index=70 + m)
    Y = orc.net_points(p, m, C)
    gamma = 1.0 / np.arange(1, s + 1) ** 1.5
    f = orc.eval_product(p, m, Y, 0.3 + 0.1 * np.arange(s))
    r = orc.spline(p, m, Y, f, alpha, gamma)
    Kmat = _kernel_matrix(orc, p, m, Y, alpha, gamma, orc.kprime)
    c = np.linalg.solve(Kmat, f)
    assert np.allclose(r["c"].real, c, rtol=1e-9, atol=1e-11 * np.abs(c).max())
    assert np.abs(r["c"].imag).max() < 1e-9 * np.abs(c).max()
    assert np.allclose(Kmat @ r["c"].real, f, rtol=1e-10)


@pytest.mark.parametrize("p,m,s,alpha", [(2, 5, 3, 2.0), (3, 3, 3, 2.0), (2, 4, 4, 1.5)])
def test_variances_equal_double_sums(orc, p, m, s, alpha):
    C = S.small_net(p, m, s, index=80 + m)
    Y = orc.net_points(p, m, C)
    gamma = 0.8 / np.arange(1, s + 1)
    f = orc.eval_exp(p, m, Y)
    r = orc.spline(p, m, Y, f, alpha, gamma)
    c = r["c"].real
    N = p ** m
    # R'(x_{n,j} (-) x_{v,j}, 0) for every pair and coordinate
    Rp = np.empty((s, N, N))
    for j in range(s):
        for n in range(N):
            for v in range(N):
                Rp[j, n, v] = orc.rprime(p, m, alpha, _dsub(int(Y[j, n]), int(Y[j, v]), p, m))
    var_u = {}
    for size in range(1, s + 1):
        for u in itertools.combinations(range(s), size):
            Ru = np.ones((N, N))
            for j in u:
                Ru *= gamma[j] ** 2 * Rp[j]
            var_u[u] = float(c @ Ru @ c)
    vt = [sum(v for u, v in var_u.items() if max(u) < d) for d in range(s + 1)]
    vs = [sum(v for u, v in var_u.items() if len(u) <= d) for d in range(s + 1)]
    tot = vt[-1]
    assert np.allclose(r["var_trc"], vt, rtol=1e-9, atol=1e-12 * tot)
    assert np.allclose(r["var_sup"], vs, rtol=1e-9, atol=1e-12 * tot)
    dt, ds = orc.effdim_threshold(np.array(vt), np.array(vs))
    assert (r["d_trc"], r["d_sup"]) == (dt, ds)


def _dadd(a, b, p, M):
    return sum(((((a // p ** i) % p) + ((b // p ** i) % p)) % p) * p ** i for i in range(M))


@pytest.mark.parametrize("p,m,s,M", [(2, 5, 3, 6), (2, 4, 2, 7), (3, 3, 2, 4), (5, 2, 3, 3), (2, 5, 3, 5)])
def test_spline_values_at_shifted_points(orc, p, m, s, M):
    """Sf(x_n (+) delta) by the DWT route against the direct sum over the net, with
    K(x (-) x_v, 0) from the short form on M digits; delta with M digits (for
    p = 2, M = m + 1 is the second half of a 2^(m+1)-point net)."""
    C = S.small_net(p, m, s, index=120 + m)
    Y = orc.net_points(p, m, C)
    gamma = 0.7 / np.arange(1, s + 1)
    alpha = 2.0
    f = orc.eval_product(p, m, Y, 0.4 + 0.1 * np.arange(s))
    c = orc.spline(p, m, Y, f, alpha, gamma)["c"].real
    delta = S.integers(S.stream_seed(61, S.P_SAMPLE, m), s, 0, p ** M - 1).astype(np.uint32)
    got = orc.spline_values_shifted(p, m, Y, c, delta, M, alpha, gamma)
    N = p ** m
    up = p ** (M - m)
    ref = np.zeros(N)
    for n in range(N):
        for v in range(N):
            k = 1.0
            for j in range(s):
                xs = _dadd(int(Y[j, n]) * up, int(delta[j]), p, M)
                k *= 1.0 + gamma[j] * orc.kprime(p, M, alpha, _dsub(xs, int(Y[j, v]) * up, p, M))
            ref[n] += c[v] * k
    assert np.allclose(got.real, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    assert np.abs(got.imag).max() < 1e-10 * np.abs(ref).max()
    if np.all(delta == 0):
        assert np.allclose(got.real, f, rtol=1e-10)   # interpolation at the net itself


def _shift_points(Y, delta, p, m, M):
    up = p ** (M - m)
    s, N = Y.shape
    X = np.empty((N, s), dtype=np.uint32)
    for n in range(N):
        for j in range(s):
            X[n, j] = _dadd(int(Y[j, n]) * up, int(delta[j]), p, M)
    return X


@pytest.mark.parametrize("p,m,s,M", [(2, 5, 3, 5), (2, 4, 2, 7), (3, 3, 2, 4), (5, 2, 3, 3)])
def test_spline_eval_interpolates_and_matches_shifted_route(orc, p, m, s, M):
    """The direct sum at the net points returns f (the interpolation conditions,
    with c from the DWT solve), and at shifted points x_n (+) delta it equals the
    convolution route of spline_values_shifted."""
    C = S.small_net(p, m, s, index=140 + m)
    Y = orc.net_points(p, m, C)
    gamma = 0.8 / np.arange(1, s + 1) ** 1.5
    alpha = 2.0
    f = orc.eval_product(p, m, Y, 0.3 + 0.2 * np.arange(s))
    c = orc.spline(p, m, Y, f, alpha, gamma)["c"].real
    up = p ** (M - m)
    at_net = orc.spline_eval(p, m, Y, c, (Y.T.astype(np.uint64) * up).astype(np.uint32), M, alpha, gamma)
    assert np.allclose(at_net, f, rtol=1e-10, atol=1e-12)
    delta = S.integers(S.stream_seed(62, S.P_SAMPLE, m), s, 0, p ** M - 1).astype(np.uint32)
    got = orc.spline_eval(p, m, Y, c, _shift_points(Y, delta, p, m, M), M, alpha, gamma)
    ref = orc.spline_values_shifted(p, m, Y, c, delta, M, alpha, gamma).real
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("p,m,s,M", [(2, 4, 3, 9), (3, 3, 2, 6), (5, 2, 2, 4)])
def test_spline_eval_reproduces_kernel_sections(orc, p, m, s, M):
    """The spline of a kernel section f = K(. (-) x_v, 0) sampled on the net is
    that section itself (it lies in the span of the interpolant), so at points
    off the net the direct sum must return K(x (-) x_v, 0)."""
    C = S.small_net(p, m, s, index=150 + m)
    Y = orc.net_points(p, m, C)
    N = p ** m
    gamma = np.linspace(0.9, 0.4, s)
    alpha = 1.7
    v = N // 3
    f = np.array([np.prod([1.0 + gamma[j] * orc.kprime(p, m, alpha, _dsub(int(Y[j, n]), int(Y[j, v]), p, m))
                           for j in range(s)]) for n in range(N)])
    c = orc.spline(p, m, Y, f, alpha, gamma)["c"].real
    unit = np.zeros(N)
    unit[v] = 1.0
    assert np.allclose(c, unit, atol=1e-9)
    X = S.integers(S.stream_seed(63, S.P_SAMPLE, p), 40 * s, 0, p ** M - 1).astype(np.uint32).reshape(40, s)
    got = orc.spline_eval(p, m, Y, c, X, M, alpha, gamma)
    up = p ** (M - m)
    ref = np.array([np.prod([1.0 + gamma[j] * orc.kprime(p, M, alpha, _dsub(int(X[q, j]), int(Y[j, v]) * up, p, M))
                             for j in range(s)]) for q in range(40)])
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-12)

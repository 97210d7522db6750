"""Pins for the oracle's effective-dimension step (Sec. 4) against the paper's printed
closed-form values and a brute-force ANOVA decomposition."""
import itertools
import os

import numpy as np
import pytest

import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "multiplicative_effdim.txt")


def _rows():
    out = []
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            a, s, dt, ds, v = line.split()
            out.append((a, int(s), int(dt), int(ds), float(v)))
    return out


@pytest.mark.parametrize("a,s,dt,ds,var", _rows())
def test_paper_table_exact_columns(orc, a, s, dt, ds, var):
    """Tables 1-2 (Sec. 5.2): for f = prod (|4x-2| + a_k)/(1+a_k), sigma^2(f_u) = prod_{j in u}
    1/(3 (1+a_j)^2); the truncation variance is prod_{j<=d}(1+sigma_j^2) - 1 and the
    superposition variance sums the elementary symmetric polynomials e_1..e_d."""
    j = np.arange(1, s + 1, dtype=float)
    ak = {"1": np.ones(s), "k": j, "k^2": j ** 2}[a]
    sig = 1.0 / (3.0 * (1.0 + ak) ** 2)
    trc = np.concatenate([[0.0], np.cumprod(1.0 + sig) - 1.0])
    e = np.zeros(s + 1)
    e[0] = 1.0
    for x in sig:                     # coefficients of prod (1 + sig_j t)
        e[1:] = e[1:] + x * e[:-1]
    sup = np.concatenate([[0.0], np.cumsum(e[1:])])
    assert abs(trc[s] - var) < 5e-5
    assert abs(sup[s] - trc[s]) < 1e-12 * trc[s]
    assert orc.effdim_threshold(trc, sup, 0.99) == (dt, ds)


def test_threshold_edge_cases(orc):
    assert orc.effdim_threshold(np.zeros(4), np.zeros(4)) == (0, 0)
    assert orc.effdim_threshold([0, 0.99, 1.0], [0, 1.0, 1.0], 0.99) == (1, 1)
    assert orc.effdim_threshold([0, 0.98, 1.0], [0, 0.5, 1.0], 0.99) == (2, 2)


def _anova_variances(G):
    """Brute-force ANOVA (eq. ANOVAdef) of a function tabulated on an equal-measure grid,
    G of shape (n,)*s: returns {u: integral of |f_u|^2} for all subsets u."""
    s = G.ndim
    eff = {}
    for size in range(s + 1):
        for u in itertools.combinations(range(s), size):
            comp = tuple(a for a in range(s) if a not in u)
            fu = G.mean(axis=comp, keepdims=True) if comp else G.copy()
            for size2 in range(size):
                for v in itertools.combinations(u, size2):
                    fu = fu - eff[v]
            eff[u] = fu
    return {u: float(np.mean(np.abs(np.broadcast_to(fu, G.shape)) ** 2)) for u, fu in eff.items()}


@pytest.mark.parametrize("p,m,s", [(2, 2, 3), (3, 1, 3), (2, 3, 2)])
def test_binning_equals_anova_of_walsh_series(orc, p, m, s):
    """g = sum_H g(H) wal_{k(H)} is tabulated on the p^m grid per coordinate and
    decomposed by brute force; its truncation/superposition variances must equal
    the oracle's class sums over supp k(H)."""
    C = S.dense_matrices(p, m, s, index=4)
    if orc.rank(p, m, C) < m:
        C = S.small_net(p, m, s, index=4)
    st, kmap = orc.coset_leaders_bruteforce(p, m, C)
    assert st == 0
    N = p ** m
    v = S.uniform(S.stream_seed(16, S.P_VALUES, p), 2 * N) - 0.5
    g = v[:N] + (1j * v[N:] if p > 2 else 0)
    n1 = p ** m
    grid = np.array(list(itertools.product(range(n1), repeat=s)))     # x_j = grid / p^m
    w = np.exp(2j * np.pi / p)
    vals = np.zeros(len(grid), dtype=complex)
    for H in range(N):
        e = np.zeros(len(grid), dtype=np.int64)
        for j in range(s):
            for i in range(m):
                kd = (int(kmap[H][j]) // p ** i) % p
                xd = (grid[:, j] // p ** (m - 1 - i)) % p        # digit x_{i+1}
                e += kd * xd
        vals += g[H] * w ** (e % p)
    var = _anova_variances(vals.reshape([n1] * s))
    trc = [sum(v for u, v in var.items() if u and max(u) < d) for d in range(s + 1)]
    sup = [sum(v for u, v in var.items() if u and len(u) <= d) for d in range(s + 1)]
    _, cls = None, orc.weight_class(kmap)[2]
    vt, vs, dt, ds = orc.effdim(g, cls, s)
    assert np.allclose(vt, trc, rtol=1e-12, atol=1e-14)
    assert np.allclose(vs, sup, rtol=1e-12, atol=1e-14)
    assert (dt, ds) == orc.effdim_threshold(np.array(trc), np.array(sup))

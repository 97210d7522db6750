"""A host model of the register-group layout of the generic passes, run over
the library's own pass splits (dwt_pass_plan_for): in every group of every
pass, the tasks of a tile cover each tile element exactly once, every shared
memory index lies inside the tile's allocation, every global offset inside the
function, and the thread count stays within the launch limit.  The model
follows the kernels' numbering: tasks column first, then the low row digits
below the group (rl), then the row digits above it (rh), or rh before rl in
the middle groups for odd p; the first group takes the top digits, the others
go bottom-up."""
import numpy as np
import pytest

BUDGET = 64 * 1024


@pytest.fixture(scope="module")
def dwtlib():
    from paper_0808_0487_gb300 import build
    build.build()
    import paper_0808_0487_gb300 as dwt
    return dwt


def _kmax(p, elem):
    if p == 2:
        return 4 if elem == 8 else 5
    if elem == 8:
        return 3 if p == 3 else 2 if p == 5 else 1
    return 2 if p == 3 else 1


def _sx(e, p, elem):
    if p % 2:
        return e
    sh = 5 if elem == 4 else 4 if elem == 8 else 3
    return e + (e >> sh)


def _groups(b, km):
    k0 = min(km, b)
    g_last = 0 if b == k0 else ((b - k0 - 1) // km) * km
    out = [(b - k0, k0)]
    g0 = b - k0
    while g0 != g_last:
        g0 = 0 if g0 + out[-1][1] == b else g0 + out[-1][1]
        out.append((g0, min(km, b - k0 - g0)))
    return out, g_last


def _check_pass(p, N, elem, d0, b, wc, tiles):
    km = _kmax(p, elem)
    S, R = p ** d0, p ** b
    wlog = wc.bit_length() - 1
    nel = R * wc
    sm_elems = nel - 1 + ((nel - 1) >> (5 if elem == 4 else 4 if elem == 8 else 3)) + 1
    assert nel * elem <= BUDGET and sm_elems * elem <= 227 * 1024
    groups, g_last = _groups(b, km)
    run = p ** g_last if S == 1 else wc
    direct_out = run * elem >= 64
    k0 = groups[0][1]
    nt = min(512, max(32, -(-((R // p ** k0) * wc) // 32) * 32))
    assert nt <= 512
    nlo = -(-S // wc)
    for tile in tiles:
        lo0 = (tile % nlo) * wc
        base = lo0 + (tile // nlo) * S * R
        ncols = min(wc, S - lo0)
        assert ncols >= 1
        for gi, (g0, k) in enumerate(groups):
            first, last = gi == 0, g0 == g_last
            rhf = (p % 2 == 1) and not first and not (last and direct_out)
            nk, pg0 = p ** k, p ** g0
            pgk, nrh = pg0 * nk, R // (pg0 * nk)
            t = np.arange((R // nk) * wc, dtype=np.int64)
            c, q = t & (wc - 1), t >> wlog
            if rhf:
                rh, rl = q % nrh, q // nrh
            else:
                rl, rh = q % pg0, q // pg0
            assert (rl < pg0).all() and (rh < nrh).all()
            r0 = rl + rh * pgk
            rows = r0[:, None] + np.arange(nk)[None, :] * pg0
            assert rows.max() < R
            e = (rows << wlog) + c[:, None]
            cover = np.bincount(e.ravel(), minlength=nel)
            assert (cover == 1).all(), (p, d0, b, wc, g0, k)
            assert _sx(int(e.max()), p, elem) < sm_elems
            live = c < ncols
            offs = base + c[:, None] + S * rows
            assert offs[live].max() < N


def _cases():
    for p in (2, 3, 5, 7, 11, 13):
        for elem in (4, 8, 16):
            if p > 2 and elem == 4:
                continue
            m = 1
            while p ** m <= 2 ** 31:
                yield p, m, elem
                m += 1


def test_layout_of_every_split(dwtlib):
    rng = np.random.default_rng(7)
    n = 0
    for p, m, elem in _cases():
        N = p ** m
        d0 = 0
        for b, wc in dwtlib.dwt_pass_plan_for(p, m, elem, 304):
            S, R = p ** d0, p ** b
            ntile = -(-S // wc) * (N // (S * R))
            # first and last tiles (the ragged column chunk) and a few others
            tiles = {0, ntile - 1, -(-S // wc) - 1 if S > 1 else 0}
            tiles |= set(int(x) for x in rng.integers(0, ntile, size=3))
            _check_pass(p, N, elem, d0, b, wc, sorted(t for t in tiles if 0 <= t < ntile))
            d0 += b
            n += 1
    assert n > 400

"""The heuristic digit split of the generic passes (host only, no GPU): the
digits may be grouped into passes freely (Sec. 2.2), but the kernels need every
tile within the 64 KB shared-memory budget, power-of-2 column counts, rows of
at least 64 bytes wherever the row distance allows, and as few passes as those
limits allow."""
import pytest

BUDGET = 64 * 1024


@pytest.fixture(scope="module")
def dwtlib():
    from paper_0808_0487_gb300 import build
    build.build()
    import paper_0808_0487_gb300 as dwt
    return dwt


def _limits(p, elem):
    cap = BUDGET // elem
    wc_min = max(1, 64 // elem)
    blo = 0
    while p ** (blo + 1) <= cap:
        blo += 1
    bhi = 0
    while p ** (bhi + 1) * wc_min <= cap:
        bhi += 1
    return cap, wc_min, blo, bhi


def _cases():
    for p in (2, 3, 5, 7, 11, 13):
        m = 1
        while p ** m <= 2 ** 31:
            for elem in (4, 8, 16):
                yield p, m, elem
            m += 1


def test_split_invariants(dwtlib):
    n = 0
    for p, m, elem in _cases():
        passes = dwtlib.dwt_pass_plan_for(p, m, elem, 304)
        cap, wc_min, blo, bhi = _limits(p, elem)
        digits = [d for d, _ in passes]
        assert sum(digits) == m and all(d >= 1 for d in digits), (p, m, elem, passes)
        q_min = 1 if m <= blo else 1 + -(-(m - blo) // bhi)
        assert len(passes) == q_min, (p, m, elem, passes)
        d0 = 0
        for t, (d, wc) in enumerate(passes):
            assert wc >= 1 and wc & (wc - 1) == 0
            assert p ** d * wc <= cap, (p, m, elem, passes)
            if t == 0:
                assert wc == 1
            else:
                assert wc * elem <= 256
                # rows of at least 64 bytes wherever the pass's row distance allows them
                if p ** d0 >= wc_min:
                    assert wc >= wc_min, (p, m, elem, passes)
            d0 += d
        n += 1
    assert n > 200


@pytest.mark.parametrize("p,m,elem,want", [
    (3, 13, 8, [(8, 1), (5, 16)]),                    # the p = 3 workload: 8 + 5 digits, 128-byte rows
    (3, 16, 8, [(8, 1), (4, 32), (4, 32)]),
    (5, 10, 8, [(5, 1), (3, 32), (2, 32)]),
    (2, 25, 4, [(14, 1), (6, 64), (5, 64)]),
    (2, 31, 4, [(14, 1), (9, 32), (8, 64)]),
])
def test_known_splits(dwtlib, p, m, elem, want):
    assert dwtlib.dwt_pass_plan_for(p, m, elem, 304) == want


def test_bad_arguments(dwtlib):
    for args in ((4, 5, 8), (3, 0, 8), (3, 21, 8), (3, 5, 6)):
        with pytest.raises(dwtlib.DwtError):
            dwtlib.dwt_pass_plan_for(*args)

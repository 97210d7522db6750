"""The serving engine: continuous batching gives the same results alone and in the mix,
admits by memory, refuses when full, and matches the oracle."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


def _small_mix(n):
    reqs = []
    for r in S.serving_requests(400):
        if r["p"] ** r["m"] <= 2 ** 14 and len(reqs) < n:
            reqs.append(r)
    return reqs


def _c_len(r):
    N = r["p"] ** r["m"]
    return N if r["p"] == 2 else 2 * N


def test_alone_equals_mix(dwt):
    reqs = _small_mix(24)
    assert len({r["p"] for r in reqs}) == 3
    # alone: one slot, each request waited for before the next is submitted
    srv = dwt.dwt_server_create(0, slots=1)
    alone = []
    for r in reqs:
        c = np.empty(_c_len(r), dtype=np.float32)
        t = dwt.dwt_server_submit(srv, r["p"], r["m"], r["s"], r["C"], r["coef"], c_out=c)
        alone.append((dwt.dwt_server_wait(srv, t), c))
    srv.close()
    # in the mix: six slots, everything submitted at once
    srv = dwt.dwt_server_create(0, slots=6)
    outs = [np.empty(_c_len(r), dtype=np.float32) for r in reqs]
    tickets = [dwt.dwt_server_submit(srv, r["p"], r["m"], r["s"], r["C"], r["coef"], c_out=c)
               for r, c in zip(reqs, outs)]
    mix = [dwt.dwt_server_wait(srv, t) for t in tickets]
    srv.close()
    overlap = 0
    for k, ((ra, ca), rb, cb) in enumerate(zip(alone, mix, outs)):
        assert ra["status"] == 0 and rb["status"] == 0
        assert np.allclose(rb["var_trc"], ra["var_trc"], rtol=1e-5, atol=0)
        assert np.allclose(rb["var_sup"], ra["var_sup"], rtol=1e-5, atol=0)
        assert (rb["d_trc"], rb["d_sup"]) == (ra["d_trc"], ra["d_sup"])
        assert np.allclose(cb, ca, rtol=1e-5, atol=1e-6 * np.abs(ca).max())
        # requests admitted while an earlier one was still running
        if any(mix[j]["t_done"] > rb["t_admit"] for j in range(k)):
            overlap += 1
    assert overlap >= 6


def test_matches_oracle(dwt, orc):
    mix = _small_mix(40)
    reqs = [r for q in (2, 3, 5) for r in [x for x in mix if x["p"] == q][:2]]
    srv = dwt.dwt_server_create(0, slots=3)
    outs = [np.empty(_c_len(r), dtype=np.float32) for r in reqs]
    tickets = [dwt.dwt_server_submit(srv, r["p"], r["m"], r["s"], r["C"], r["coef"], c_out=c)
               for r, c in zip(reqs, outs)]
    for r, t, c in zip(reqs, tickets, outs):
        res = dwt.dwt_server_wait(srv, t)
        p, m, s = r["p"], r["m"], r["s"]
        f = orc.eval_product(p, m, orc.net_points(p, m, r["C"]), r["coef"])
        tab = orc.coset_leaders_dp(p, m, r["C"])
        cref, g, vt, vs, dt, ds = orc.interpolate(p, m, f, tab["W64"], tab["cls"], s)
        got = c if p == 2 else c[0::2] + 1j * c[1::2]
        ref = cref.real if p == 2 else cref
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5
        assert np.allclose(res["var_trc"], vt, rtol=1e-5, atol=1e-14 * vt[-1])
        assert np.allclose(res["var_sup"], vs, rtol=1e-5, atol=1e-14 * vt[-1])
    srv.close()


def test_admission_limits(dwt):
    big = S.serving_requests(1)[0]
    # a budget smaller than one request: refused at submit
    srv = dwt.dwt_server_create(1 << 20, slots=1)
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt_server_submit(srv, 2, 20, 16, S.small_net(2, 20, 16), np.full(16, 0.5))
    assert e.value.status == dwt.DWT_ENOMEM
    srv.close()
    # a full queue: refused with EBUSY
    srv = dwt.dwt_server_create(0, slots=1, max_queue=2)
    C = S.small_net(2, 22, 48, index=3)
    dwt.dwt_server_submit(srv, 2, 22, 48, C, np.full(48, 0.5))
    statuses = []
    for _ in range(6):
        try:
            dwt.dwt_server_submit(srv, big["p"], big["m"], big["s"], big["C"], big["coef"])
            statuses.append(0)
        except dwt.DwtError as ex:
            statuses.append(ex.status)
    assert dwt.DWT_EBUSY in statuses
    srv.close()


def test_larger_requests_complete(dwt):
    """One request of every (p, size class) of the serving mix, run concurrently."""
    picked = {}
    for r in S.serving_requests(600):
        key = (r["p"], r["m"])
        if key not in picked:
            picked[key] = r
    reqs = sorted(picked.values(), key=lambda r: r["p"] ** r["m"])
    srv = dwt.dwt_server_create(0, slots=8)
    tickets = [dwt.dwt_server_submit(srv, r["p"], r["m"], r["s"], r["C"], r["coef"]) for r in reqs]
    res = [dwt.dwt_server_wait(srv, t) for t in tickets]
    srv.close()
    bad = [(r["p"], r["m"], r["s"], x["status"], x["message"]) for r, x in zip(reqs, res) if x["status"]]
    assert not bad, bad

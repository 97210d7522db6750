"""The measured choice of the pass split (DWT_PLAN_TUNE): any grouping of the
digits gives the same transform (Sec. 2.2), so a tuned plan must match the
oracle like the heuristic one; the choice is cached in a file across
processes."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import synthetic as S
from conftest import rel_l2

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cplx(a):
    return a[0::2] + 1j * a[1::2]


@pytest.mark.parametrize("p,m", [(3, 12), (5, 7), (2, 15), (7, 6)])
def test_tuned_plan_matches_oracle(dwt, dev, orc, p, m, tmp_path, monkeypatch):
    monkeypatch.setenv("DWT_TUNE_CACHE", str(tmp_path / "tune.jsonl"))
    N = p ** m
    C = S.small_net(p, m, 2, index=40 + m)
    plan = dwt.dwt_plan_create(p, m, 2, C, dwt.DWT_PLAN_TRANSFORM_ONLY | dwt.DWT_PLAN_TUNE)
    passes = dwt.dwt_plan_passes(plan, 4 if p == 2 else 8)
    assert sum(d for d, _ in passes) == m and passes[0][1] == 1
    assert all(w >= 1 and (w & (w - 1)) == 0 for _, w in passes)
    f = orc.eval_exp(p, m, orc.net_points(p, m, C))
    fin = torch.tensor(f.astype(np.float32), device=dev)
    if p == 2:
        out = torch.empty(N, device=dev)
        dwt.dwt_forward(plan, fin, out, 1, N, N, dwt.DWT_F32, dwt.DWT_F32)
        assert rel_l2(out.cpu().numpy(), orc.fwt(p, m, f).real) < 1e-5
    else:
        out = torch.empty(2 * N, device=dev)
        dwt.dwt_forward(plan, fin, out, 1, N, N, dwt.DWT_F32, dwt.DWT_C64)
        assert rel_l2(_cplx(out.cpu().numpy()), orc.fwt(p, m, f)) < 1e-5


_CHILD = r"""
import sys, json
sys.path.insert(0, %r)
import paper_0808_0487_gb300 as dwt
import synthetic as S
p, m = 3, 11
plan = dwt.dwt_plan_create(p, m, 2, S.small_net(p, m, 2, index=5), dwt.DWT_PLAN_TRANSFORM_ONLY | dwt.DWT_PLAN_TUNE)
print(json.dumps(dwt.dwt_plan_passes(plan, 8)))
"""


def test_tune_cache_file_across_processes(tmp_path):
    cache = tmp_path / "tune.jsonl"
    env = dict(os.environ, DWT_TUNE_CACHE=str(cache))
    runs = [subprocess.run([sys.executable, "-c", _CHILD % ROOT], env=env, capture_output=True, text=True,
                           timeout=300) for _ in range(2)]
    for r in runs:
        assert r.returncode == 0, r.stderr
    first, second = (json.loads(r.stdout.strip().splitlines()[-1]) for r in runs)
    assert first == second                       # the second process read the first one's choice
    lines = [json.loads(x) for x in cache.read_text().splitlines() if x.strip()]
    mine = [x for x in lines if x["p"] == 3 and x["m"] == 11 and x["elem"] == 8]
    assert len(mine) == 1                        # measured once
    assert mine[0]["digits"] == [d for d, _ in first] and mine[0]["wc"] == [w for _, w in first]


@pytest.mark.parametrize("p,m", [(2, 17), (2, 18), (3, 9)])
def test_tuned_choices_keep_results(dwt, dev, orc, p, m, tmp_path, monkeypatch):
    """The measured launch choices (p = 2 low-pass digits, tensor-core form for
    DWT_ALGO_AUTO, functions per L2 group) leave the transform within the same
    tolerance of the oracle, and are reported in the kernels' ranges."""
    monkeypatch.setenv("DWT_TUNE_CACHE", str(tmp_path / "tune.jsonl"))
    N = p ** m
    C = S.small_net(p, m, 2, index=60 + m)
    plan = dwt.dwt_plan_create(p, m, 2, C, dwt.DWT_PLAN_TRANSFORM_ONLY | dwt.DWT_PLAN_TUNE)
    ch = dwt.dwt_plan_tuned(plan)
    if p == 2 and m <= 19:
        assert max(12, m - 10) <= ch["lo_digits"] <= min(14, m - 4)
    else:
        assert ch["lo_digits"] == 0
    assert ch["tc"] in (0, 1) and (ch["tc"] == 0 or (p == 2 and (m == 14 or 18 <= m <= 24)))
    assert ch["group_bytes"] in (0, 16 << 20, 128 << 20, 1024 << 20)
    line = [json.loads(x) for x in (tmp_path / "tune.jsonl").read_text().splitlines() if x.strip()][-1]
    assert line["lo"] == ch["lo_digits"] and line["tc"] == ch["tc"] and line["group_mb"] << 20 == ch["group_bytes"]
    f = orc.eval_exp(p, m, orc.net_points(p, m, C))
    fin = torch.tensor(np.tile(f.astype(np.float32), (3, 1)), device=dev)
    if p == 2:
        out = torch.empty((3, N), device=dev)
        dwt.dwt_forward(plan, fin, out, 3, N, N, dwt.DWT_F32, dwt.DWT_F32)
        ref = orc.fwt(p, m, f).real
        for b in range(3):
            assert rel_l2(out[b].cpu().numpy(), ref) < 1e-5
        back = torch.empty_like(out)
        dwt.dwt_inverse(plan, out, back, 3, N, N, dwt.DWT_F32, dwt.DWT_F32)
        assert rel_l2(back[0].cpu().numpy(), f) < 1e-5
    else:
        out = torch.empty((3, 2 * N), device=dev)
        dwt.dwt_forward(plan, fin, out, 3, N, N, dwt.DWT_F32, dwt.DWT_C64)
        assert rel_l2(_cplx(out[2].cpu().numpy()), orc.fwt(p, m, f)) < 1e-5

"""The structs of the C ABI (include/dwt.h) and their ctypes mirrors in the
Python binding have the same size and field offsets (checked by compiling a
probe against the header with the host C compiler; no GPU), and the grouped
transform refuses an empty job list before any device work."""
import ctypes
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_PROBE = r"""
#include <stdio.h>
#include <stddef.h>
#include "dwt.h"
#define F(T, f) printf("%s.%s %zu\n", #T, #f, offsetof(T, f))
int main(void) {
    printf("dwt_job %zu\n", sizeof(dwt_job));
    F(dwt_job, plan); F(dwt_job, in); F(dwt_job, out); F(dwt_job, batch); F(dwt_job, ld_in); F(dwt_job, ld_out);
    printf("dwt_request %zu\n", sizeof(dwt_request));
    F(dwt_request, p); F(dwt_request, m); F(dwt_request, s); F(dwt_request, C); F(dwt_request, coef);
    F(dwt_request, weight); F(dwt_request, threshold); F(dwt_request, c_out);
    printf("dwt_result %zu\n", sizeof(dwt_result));
    F(dwt_result, status); F(dwt_result, s); F(dwt_result, d_trc); F(dwt_result, d_sup); F(dwt_result, var_trc);
    F(dwt_result, var_sup); F(dwt_result, t_submit); F(dwt_result, t_done); F(dwt_result, message);
    return 0;
}
"""


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    d = tmp_path_factory.mktemp("abi")
    src = d / "probe.c"
    src.write_text(_PROBE)
    exe = d / "probe"
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("no host C compiler: " + r.stderr[:200])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


def _py_layout(cls, cname, fields):
    got = {cname: ctypes.sizeof(cls)}
    for py, c in fields:
        got["%s.%s" % (cname, c)] = getattr(cls, py).offset
    return got


def test_struct_layouts_match(c_layout):
    import paper_0808_0487_gb300 as dwt
    got = {}
    got.update(_py_layout(dwt._Job, "dwt_job", [("plan", "plan"), ("in_", "in"), ("out", "out"), ("batch", "batch"),
                                                 ("ld_in", "ld_in"), ("ld_out", "ld_out")]))
    got.update(_py_layout(dwt.dwt_request, "dwt_request",
                          [(f, f) for f in ("p", "m", "s", "C", "coef", "weight", "threshold", "c_out")]))
    got.update(_py_layout(dwt.dwt_result, "dwt_result",
                          [(f, f) for f in ("status", "s", "d_trc", "d_sup", "var_trc", "var_sup", "t_submit",
                                            "t_done", "message")]))
    assert got == c_layout


def test_grouped_rejects_empty_list_without_a_device():
    from paper_0808_0487_gb300 import build
    build.build()
    import paper_0808_0487_gb300 as dwt
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt_forward_grouped([], dwt.DWT_F32, dwt.DWT_F32)
    assert e.value.status == dwt.DWT_EINVAL
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt_inverse_grouped([], dwt.DWT_F32, dwt.DWT_F32)
    assert e.value.status == dwt.DWT_EINVAL

"""The C-ABI library builds, loads and exports every entry point of include/dwt.h;
host-side argument checks work without a GPU (no compute call is made)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dwt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(dwt_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def dwtlib():
    from paper_0808_0487_gb300 import build
    build.build()
    import paper_0808_0487_gb300 as dwt
    return dwt


def test_every_declared_symbol_is_exported(dwtlib):
    names = _declared()
    assert len(names) >= 19
    L = ctypes.CDLL(dwtlib.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding exposes the same names
    assert all(hasattr(dwtlib, n) for n in names)


def test_strerror_and_host_checks(dwtlib):
    assert dwtlib.dwt_strerror(0) == "ok"
    assert "span" in dwtlib.dwt_strerror(dwtlib.DWT_ESPAN)
    C = np.zeros((1, 3, 3), dtype=np.uint8)
    with pytest.raises(dwtlib.DwtError) as e:          # p = 4 is not prime
        dwtlib.dwt_plan_create(4, 3, 1, C)
    assert e.value.status == dwtlib.DWT_EINVAL
    C[0, 0, 0] = 2                                      # entry >= p
    with pytest.raises(dwtlib.DwtError) as e:
        dwtlib.dwt_plan_create(2, 3, 1, C)
    assert e.value.status == dwtlib.DWT_EINVAL
    with pytest.raises(dwtlib.DwtError):                # p^m > 2^31
        dwtlib.dwt_plan_create(2, 32, 1, np.zeros((1, 32, 32), dtype=np.uint8))


def test_plan_and_plan_create_are_one_call(dwtlib):
    """dwt_plan is the plan call of the boundary; dwt_plan_create keeps the same
    behaviour (here: the host-side argument checks, no device work)."""
    for bad in ((4, 3, 1, np.zeros((1, 3, 3), dtype=np.uint8)),      # p not prime
                (2, 3, 1, np.full((1, 3, 3), 2, dtype=np.uint8)),     # entry >= p
                (2, 3, 0, np.zeros((0, 3, 3), dtype=np.uint8))):      # s < 1
        for call in (dwtlib.dwt_plan, dwtlib.dwt_plan_create):
            with pytest.raises(dwtlib.DwtError) as e:
                call(*bad)
            assert e.value.status == dwtlib.DWT_EINVAL


def test_no_cpu_fallback_in_package():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_0808_0487_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "oracle.c" not in txt, f


def test_missing_library_fails_loudly(dwtlib, monkeypatch, tmp_path):
    """Without the built library every call raises: there is no other path."""
    monkeypatch.setattr(dwtlib, "_lib", None)
    monkeypatch.setattr(dwtlib, "LIB_PATH", str(tmp_path / "libdwt.so"))
    with pytest.raises(dwtlib.DwtError):
        dwtlib.dwt_strerror(0)
    with pytest.raises(dwtlib.DwtError):
        dwtlib.dwt_plan_create(2, 4, 1, np.zeros((1, 4, 4), dtype=np.uint8))

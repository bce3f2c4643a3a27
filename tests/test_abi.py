"""The C-ABI library: it loads, exports every symbol include/mbbp.h declares,
and its host-only steps (Algorithm 2, root orders, the subtree collection)
agree exactly with the oracle.  No CUDA call is made here."""
import os
import re

import numpy as np
import pytest

import oracle
from conftest import ROOT
from paper_2605_14170_gb300.inputs import named_code


@pytest.fixture(scope="module")
def lib():
    from paper_2605_14170_gb300 import build
    build.build()
    from paper_2605_14170_gb300 import mbbp
    return mbbp


def declared_functions():
    names = []
    for fname in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fname.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fname)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(mbbp_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib._lib, name), name
        assert name in lib.EXPORTED, f"{name} has no binding"


def test_version_and_error_string(lib):
    assert "sm_103a" in lib.mbbp_version()
    with pytest.raises(lib.MBBPError):
        lib.mbbp_permutation(1, -1, 4)
    assert "bad arguments" in lib.mbbp_last_error()


def test_probe_rejects_bad_arguments(lib):
    """The throughput probe checks its arguments before any CUDA call."""
    import ctypes as C
    work = C.c_double(0.0)
    assert lib._lib.mbbp_probe(9, 1, None, C.byref(work), None) == 1
    assert "unknown kind" in lib.mbbp_last_error()
    assert lib._lib.mbbp_probe(lib.PROBE_FADD, 0, None, C.byref(work), None) == 1


def test_fig2_example_host(lib):
    H = np.array([[1, 1, 1, 0, 0, 0], [0, 1, 1, 0, 0, 1], [1, 0, 0, 1, 1, 0], [0, 0, 0, 1, 1, 1]], np.uint8)
    cs, order, ns = lib.mbbp_subtrees(H, np.array([0, 3, 1, 2]))
    assert ns == 2 and cs.tolist() == [1, 2, 1, 2] and order.tolist() == [0, 2, 3, 1]


@pytest.mark.parametrize("code", ["bb72", "bb144", "bb288", "gb882"])
def test_subtrees_match_oracle(lib, code):
    c = named_code(code)
    for H in (c.HX, c.HZ):
        m = H.shape[0]
        for j in range(4):
            perm = lib.mbbp_permutation(5, j, m)
            assert np.array_equal(perm, oracle.permutation(5, j, m))
            a = lib.mbbp_subtrees(H, perm)
            b = oracle.subtrees(H, perm)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
        R = 64 if code == "gb882" else 16
        got = lib.mbbp_collect_subtrees(H, R, 20260514)
        ref = oracle.collect_subtrees(H, R, 20260514)
        assert len(got) == len(ref) == R
        assert all(np.array_equal(x, y) for x, y in zip(got, ref))


def test_random_graphs_match_oracle(lib):
    rng = np.random.default_rng(3)
    for _ in range(50):
        m, n = rng.integers(2, 30), rng.integers(3, 40)
        H = (rng.random((m, n)) < 0.2).astype(np.uint8)
        perm = rng.permutation(m).astype(np.int32)
        a, b = lib.mbbp_subtrees(H, perm), oracle.subtrees(H, perm)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_invalid_host_arguments(lib):
    H = np.ones((3, 4), np.uint8)
    with pytest.raises(lib.MBBPError):
        lib.mbbp_subtrees(H, np.array([0, 0, 1]))  # not a permutation
    with pytest.raises(lib.MBBPError):
        lib.mbbp_subtrees(np.full((3, 4), 2, np.uint8), np.array([0, 1, 2]))
    with pytest.raises(lib.MBBPError):
        lib.mbbp_collect_subtrees(H, 65, 1)
    tiny = np.array([[1, 1, 0], [0, 1, 1]], np.uint8)
    with pytest.raises(lib.MBBPError) as err:
        lib.mbbp_collect_subtrees(tiny, 5, 1)
    assert err.value.status == 6  # MBBP_E_NOT_FOUND


def test_missing_library_fails_loudly(tmp_path):
    """The binding raises instead of falling back when libmbbp.so is absent."""
    import shutil
    import subprocess
    import sys
    pkg = os.path.join(ROOT, "paper_2605_14170_gb300")
    dst = tmp_path / "paper_2605_14170_gb300"
    dst.mkdir()
    for f in ("__init__.py", "mbbp.py"):
        shutil.copy(os.path.join(pkg, f), dst / f)
    res = subprocess.run([sys.executable, "-c", "import paper_2605_14170_gb300.mbbp"],
                         cwd=tmp_path, capture_output=True, text=True)
    assert res.returncode != 0 and "is not built" in res.stderr


def test_random_sets_host_equals_oracle(lib):
    """Random augmentation (Table II): the library's sets equal the oracle's."""
    for m, sizes, seed in ((72, [3, 9, 1, 0, 72, 80], 5), (441, [40] * 64, 123), (1, [1, 0, 2], 9)):
        a = lib.mbbp_random_sets(m, sizes, seed)
        b = oracle.random_sets(m, sizes, seed)
        assert [x.tolist() for x in a] == [x.tolist() for x in b]
    with pytest.raises(lib.MBBPError):
        lib.mbbp_random_sets(10, [-1], 1)


def test_workspace_size_queries_reject_bad_arguments(lib):
    """Every size query answers 0 for a NULL handle (and the WMS ones for a
    negative batch or T < 1) before touching a device."""
    L = lib._lib
    assert L.mbbp_decode_workspace_size(None, 10) == 0
    assert L.mbbp_wms_workspace_size(None, 10, 25, 5) == 0
    assert L.mbbp_wms_decode_workspace_size(None, 10, 25) == 0
    assert L.mbbp_plan_workspace_size(None, np.zeros(1, np.int32)) == 0

"""The C ABI boundary: libegs.so builds for sm_103a, loads without a GPU, and
exports every function include/egs.h declares.  Only host-side queries are
called here (no kernel runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "egs.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(egs_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1708_02835_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("egs_matern_tiles", "egs_loglik", "egs_loglik_batched", "egs_serve_create", "egs_serve_submit",
                     "egs_serve_wait", "egs_serve_stats", "egs_serve_destroy", "egs_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    handle, path = lib
    missing = [n for n in _declared() if not hasattr(handle, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (egs_[a-z0-9_]+)", out))
    assert set(_declared()) <= exported


def test_host_only_queries(lib):
    import paper_1708_02835_gb300 as egs
    egs.load_library()
    assert egs.egs_version().startswith("egs")
    assert egs.egs_default_tile(1600, "fp64") == 128
    assert egs.egs_default_tile(102400, "tf32") == 512
    # 200 x 201 / 2 tiles of 512 x 512 doubles
    assert egs.egs_tiles_bytes(102400, 512, "fp64") == 20100 * 512 * 512 * 8
    assert egs.egs_tiles_bytes(100, 100, "fp64") == 0          # tile must be a multiple of 64
    # a mixed evaluation holds its own tile storage but no FP64 copy of Sigma (the
    # refinement regenerates it): less than the FP64 tiles alone
    ws = egs.egs_loglik_workspace_bytes(102400, 512, "tf32", 2)
    assert egs.egs_tiles_bytes(102400, 512, "tf32", 2) < ws < egs.egs_tiles_bytes(102400, 512, "fp64")
    assert egs.egs_loglik_workspace_bytes(1000, 320, "tf32", 2) == 0   # mixed needs tile % 256 == 0
    # mixed storage: 200 x 3 band tiles of doubles + 197 x 198 / 2 off-band tiles of floats
    assert egs.egs_tiles_bytes(102400, 512, "fp32", 3) == 600 * 512 * 512 * 8 + 19503 * 512 * 512 * 4
    assert egs.egs_tiles_bytes(1024, 512, "fp32", 2) == egs.egs_tiles_bytes(1024, 512, "fp64")  # T <= band


def test_built_for_sm103a_only():
    from paper_1708_02835_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_trace_is_empty_before_any_traced_call(lib):
    import paper_1708_02835_gb300 as egs
    assert egs.egs_trace_last() == []
    handle, _ = lib
    handle.egs_trace_last.restype = ctypes.c_int
    assert handle.egs_trace_last(None, ctypes.c_int64(0), None) == 1        # EGS_ERR_ARG: count is NULL
    cnt = ctypes.c_int64(-1)
    assert handle.egs_trace_last(None, ctypes.c_int64(4), ctypes.byref(cnt)) == 1   # NULL out with cap > 0

"""Host-side argument checks of the C ABI: failure detection by fault
injection on the host (NaN, infinite, zero or negative theta; empty or
oversized requests; bad tiles, precisions and options; a zero serving budget).
Every call here is rejected before any device work, so these run without a
GPU; the library must answer with a status code and a message (no abort, no
print), and egs_loglik_ex must leave NaN in its output."""
import ctypes
import math

import numpy as np
import pytest

import paper_1708_02835_gb300 as egs

N = 100
LOCS = np.zeros(2 * N)
Z = np.zeros(N)
GOOD = (1.0, 0.1, 0.5)


@pytest.fixture(scope="module", autouse=True)
def lib():
    return egs.load_library()


def _status(fn, *args, **kw):
    with pytest.raises(egs.EgsError) as e:
        fn(*args, **kw)
    assert egs.egs_last_error() != ""
    return e.value.status, str(e.value)


@pytest.mark.parametrize("theta", [(float("nan"), 0.1, 0.5), (1.0, -0.1, 0.5), (1.0, 0.1, float("inf")),
                                   (0.0, 0.1, 0.5), (1.0, 0.1, -math.inf)])
def test_theta_must_be_finite_and_positive(theta):
    st, msg = _status(egs.egs_loglik_ex, LOCS, Z, theta, N, "fp64")
    assert st == egs.EGS_ERR_ARG and "theta" in msg
    st, _ = _status(egs.egs_loglik_ind, LOCS, Z, theta, N, 64, 1)
    assert st == egs.EGS_ERR_ARG
    st, _ = _status(egs.egs_matern_tiles, LOCS, N, theta, 64, np.zeros(4))
    assert st == egs.EGS_ERR_ARG


def test_output_is_nan_on_failure(lib):
    th = (ctypes.c_double * 3)(float("nan"), 0.1, 0.5)
    out = ctypes.c_double(123.0)
    st = lib.egs_loglik_ex(LOCS.ctypes.data, Z.ctypes.data, th, N, 0, None, ctypes.byref(out), None, None)
    assert st == egs.EGS_ERR_ARG and math.isnan(out.value)


def test_sizes_tiles_and_precisions():
    assert _status(egs.egs_loglik_ex, LOCS, Z, GOOD, 0, "fp64")[0] == egs.EGS_ERR_ARG            # n = 0
    assert _status(egs.egs_loglik_ex, LOCS, Z, GOOD, N, "fp64", tile=100)[0] == egs.EGS_ERR_ARG  # not % 64
    assert _status(egs.egs_loglik_ex, LOCS, Z, GOOD, N, "fp64", tile=2048)[0] == egs.EGS_ERR_ARG
    st, msg = _status(egs.egs_loglik_ex, LOCS, Z, GOOD, N, "fp32", tile=320)                    # mixed: % 256
    assert st == egs.EGS_ERR_ARG and "256" in msg
    assert _status(egs.egs_loglik_ex, LOCS, Z, GOOD, N, 9)[0] == egs.EGS_ERR_UNIMPLEMENTED
    assert _status(egs.egs_matern_tiles, LOCS, 0, GOOD, 64, np.zeros(4))[0] == egs.EGS_ERR_ARG
    assert _status(egs.egs_matern_tiles, LOCS, N, GOOD, 64, np.zeros(4), 9)[0] == egs.EGS_ERR_UNIMPLEMENTED
    assert _status(egs.egs_loglik_ind, LOCS, Z, GOOD, N, 64, 0)[0] == egs.EGS_ERR_ARG           # super_tiles = 0
    assert _status(egs.egs_loglik_ind, LOCS, Z, GOOD, N, 100, 1)[0] == egs.EGS_ERR_ARG
    z_new = np.zeros(4)
    assert _status(egs.egs_predict, LOCS, Z, N, np.zeros(8), 0, GOOD, z_new)[0] == egs.EGS_ERR_ARG  # m = 0


def test_options_are_checked(lib):
    th = (ctypes.c_double * 3)(*GOOD)
    out = ctypes.c_double()
    opts = egs.egs_opts(distance=5)
    st = lib.egs_loglik_ex(LOCS.ctypes.data, Z.ctypes.data, th, N, 0, ctypes.byref(opts), ctypes.byref(out), None,
                           None)
    assert st == egs.EGS_ERR_ARG and "distance" in egs.egs_last_error()
    opts = egs.egs_opts(band=3, xband=2)
    st = lib.egs_loglik_ex(LOCS.ctypes.data, Z.ctypes.data, th, N, 1, ctypes.byref(opts), ctypes.byref(out), None,
                           None)
    assert st == egs.EGS_ERR_ARG and "xband" in egs.egs_last_error()
    need = egs.egs_loglik_workspace_bytes(N, 64, "fp64", 2)
    assert need > 0
    small = np.zeros(16, dtype=np.uint8)
    opts = egs.egs_opts(tile=64, workspace=small.ctypes.data, workspace_bytes=small.nbytes)
    st = lib.egs_loglik_ex(LOCS.ctypes.data, Z.ctypes.data, th, N, 0, ctypes.byref(opts), ctypes.byref(out), None,
                           None)
    assert st == egs.EGS_ERR_ARG and "workspace" in egs.egs_last_error()


def test_batches_and_servers():
    assert _status(egs.egs_batch, [])[0] == egs.EGS_ERR_ARG
    assert _status(egs.egs_batch, [100, 200], 0, "tf32")[0] == egs.EGS_ERR_UNIMPLEMENTED
    assert _status(egs.egs_batch, [100, 200], 100)[0] == egs.EGS_ERR_ARG
    assert _status(egs.egs_server, 0)[0] == egs.EGS_ERR_ARG                                     # zero budget
    assert _status(egs.egs_server, 1 << 30, max_inflight=0)[0] == egs.EGS_ERR_ARG
    assert _status(egs.egs_server, 1 << 30, max_inflight=65)[0] == egs.EGS_ERR_ARG


def test_solves_reject_host_pointers():
    """The factor, right-hand side and solution of the tile solves (and the
    tiles of the factorisation and the generator) are device memory; host
    arrays are answered with EGS_ERR_ARG before any kernel sees them."""
    tiles = np.zeros(64 * 64)
    z, y = np.zeros(64), np.zeros(64)
    for fn in (egs.egs_trsv_tiles, egs.egs_trsv_tiles_noalloc):
        st, msg = _status(fn, tiles, 64, 64, z, y)
        assert st == egs.EGS_ERR_ARG and "device" in msg
    st, msg = _status(egs.egs_potrf_tiles, tiles, 64, 64)
    assert st == egs.EGS_ERR_ARG and "device" in msg
    st, msg = _status(egs.egs_matern_tiles, np.zeros(128), 64, GOOD, 64, tiles)
    assert st == egs.EGS_ERR_ARG and "device" in msg


def test_withheld_stage_must_be_a_stage():
    a = np.zeros((128, 64), dtype=np.float32)
    b = np.zeros((256, 64), dtype=np.float32)
    c = np.zeros((128, 256), dtype=np.float32)
    st, msg = _status(egs.egs_tc_gemm_test_withhold, a, b, c, "tf32", -1)
    assert st == egs.EGS_ERR_ARG and "withhold" in msg

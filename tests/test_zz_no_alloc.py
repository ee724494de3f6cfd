"""egs_trsv_tiles_noalloc: the forward solve for callers that cannot
allocate device memory during the call (its scratch is a fixed device array
inside the library).  Checked against egs_trsv_tiles, which allocates its
scratch per call, on two calls in a row (the second call reuses the array the
first one left behind), plus the size limit.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import egs_inputs as ei

pytestmark = pytest.mark.gpu


def _factor(egs, n, tile, theta, seed):
    import torch
    locs = ei.jittered_grid(n, seed=seed)
    dl = torch.as_tensor(np.ascontiguousarray(locs.reshape(-1))).cuda()
    tiles = torch.empty(egs.egs_tiles_bytes(n, tile) // 8, dtype=torch.float64, device="cuda")
    egs.egs_matern_tiles(dl, n, theta, tile, tiles)
    assert egs.egs_potrf_tiles(tiles, n, tile) == -1
    return tiles


@pytest.mark.parametrize("n,tile", [(1000, 128), (3001, 256)])
def test_noalloc_matches_allocating_solve_twice(n, tile):
    import torch
    import paper_1708_02835_gb300 as egs
    egs.load_library()
    tiles = _factor(egs, n, tile, (1.0, 0.1, 0.5), seed=4)
    for call in range(2):
        z = torch.as_tensor(ei.normal(50 + call, n)).cuda()
        y_ref = torch.empty_like(z)
        ld_ref, q_ref = egs.egs_trsv_tiles(tiles, n, tile, z, y_ref)
        y = torch.full_like(z, float("nan"))
        ld, q = egs.egs_trsv_tiles_noalloc(tiles, n, tile, z, y)
        torch.cuda.synchronize()
        assert torch.allclose(y, y_ref, rtol=1e-12, atol=0.0)
        assert abs(ld - ld_ref) <= 1e-12 * abs(ld_ref)
        assert abs(q - q_ref) <= 1e-12 * abs(q_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_1708_02835_gb300 as egs
    egs.load_library()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(egs.EgsError) as e:
        egs.egs_trsv_tiles_noalloc(dummy, 200000, 512, dummy, dummy)
    assert e.value.status == egs.EGS_ERR_ARG and "scratch" in str(e.value)
    # a successful call after the rejected one leaves no stale message behind
    n, tile = 500, 128
    tiles = _factor(egs, n, tile, (1.0, 0.1, 0.5), seed=6)
    z = torch.as_tensor(ei.normal(60, n)).cuda()
    y = torch.empty_like(z)
    egs.egs_trsv_tiles_noalloc(tiles, n, tile, z, y)
    assert egs.egs_last_error() == ""


def test_noalloc_rejects_host_pointers():
    import torch
    import paper_1708_02835_gb300 as egs
    egs.load_library()
    n, tile = 500, 128
    tiles = _factor(egs, n, tile, (1.0, 0.1, 0.5), seed=6)
    z = ei.normal(61, n)
    y = np.empty(n)
    with pytest.raises(egs.EgsError) as e:
        egs.egs_trsv_tiles_noalloc(tiles, n, tile, z, y)
    assert e.value.status == egs.EGS_ERR_ARG and "device" in str(e.value)

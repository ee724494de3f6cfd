"""The caller-supplied allocator hook on the GPU: evaluations, the
allocation-heavy calls and the serving loop take their device memory from
the caller (here PyTorch tensors, and PyTorch's caching allocator) and give
the same results, bit for bit, as with the library's own cudaMallocAsync;
every allocation is returned."""
import numpy as np
import pytest

import egs_inputs as ei
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture()
def egs():
    import paper_1708_02835_gb300 as m
    m.load_library()
    yield m
    m.egs_set_allocator(None, None)


class TensorPool:
    """alloc / free hooks that hand out torch tensors and record the calls."""

    def __init__(self):
        import torch
        self.torch = torch
        self.live = {}
        self.calls = []

    def alloc(self, nbytes, stream):
        t = self.torch.empty(max(nbytes, 1), dtype=self.torch.uint8, device="cuda")
        # the tensor's memory may have been released by work still queued on
        # this thread's stream; the library uses it on `stream`
        self.torch.cuda.current_stream().synchronize()
        self.live[t.data_ptr()] = t
        self.calls.append(("alloc", nbytes))
        return t.data_ptr()

    def free(self, ptr, nbytes, stream):
        self.calls.append(("free", nbytes))
        # the default stream orders the library's work before any later use
        del self.live[ptr]


@pytest.mark.parametrize("prec,theta", [("fp64", (1.0, 0.1, 0.5)), ("fp32", (1.0, 0.1, 0.5)),
                                        ("fp32", (1.0, 0.05, 0.8))])
def test_hook_gives_identical_evaluations(egs, prec, theta):
    from gpu_util import locs_dev, dev
    n = 3000
    p = ei.Problem(n=n, theta=theta, seed=5)
    locs = p.locations()
    z = oracle.simulate_z(locs, theta, p.e())
    ref, _ = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, prec, tile=256, band=2)
    pool = TensorPool()
    egs.egs_set_allocator(pool.alloc, pool.free)
    got, _ = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, prec, tile=256, band=2)
    egs.egs_set_allocator(None, None)
    assert got == ref
    assert pool.calls == [("alloc", egs.egs_loglik_workspace_bytes(n, 256, prec, 2)),
                          ("free", egs.egs_loglik_workspace_bytes(n, 256, prec, 2))]
    assert not pool.live


def test_torch_caching_allocator_for_every_call(egs):
    import torch
    from gpu_util import locs_dev, dev
    n, theta = 2000, (1.0, 0.1, 1.3)
    p = ei.Problem(n=n, theta=theta, seed=6)
    locs = p.locations()
    z = oracle.simulate_z(locs, theta, p.e())
    dl, dz = locs_dev(locs), dev(z)

    def run():
        out = {}
        out["l64"], _ = egs.egs_loglik_ex(dl, dz, theta, n, "fp64", tile=128)
        out["l32"], _ = egs.egs_loglik_ex(dl, dz, theta, n, "fp32", tile=256, band=2)
        zs = torch.empty(n, dtype=torch.float64, device="cuda")
        egs.egs_simulate(dl, dz, theta, n, zs, tile=128)
        out["sim"] = zs.cpu().numpy()
        tiles = torch.empty(egs.egs_tiles_bytes(n, 128) // 8, dtype=torch.float64, device="cuda")
        egs.egs_matern_tiles(dl, n, theta, 128, tiles)
        egs.egs_potrf_tiles(tiles, n, 128)
        y = torch.empty_like(dz)
        out["trsv"] = egs.egs_trsv_tiles(tiles, n, 128, dz, y)
        torch.cuda.synchronize()
        return out

    ref = run()
    egs.use_torch_allocator()
    got = run()
    egs.egs_set_allocator(None, None)
    assert got["l64"] == ref["l64"] and got["l32"] == ref["l32"] and got["trsv"] == ref["trsv"]
    assert np.array_equal(got["sim"], ref["sim"])


def test_serving_with_the_hook(egs):
    """Fields and slot workspaces come from the hook fixed at creation; served
    values equal the direct call's; everything is returned at destroy."""
    from gpu_util import locs_dev, dev
    fields = [ei.Problem(n=n, theta=(1.0, 0.1, 0.5), seed=s) for s, n in enumerate((1500, 2500))]
    ref = [egs.egs_loglik_ex(locs_dev(f.locations()), dev(f.e()), (1.0, 0.1, 0.5), f.n, "fp32", tile=256,
                             band=2)[0] for f in fields]
    pool = TensorPool()
    egs.egs_set_allocator(pool.alloc, pool.free)
    srv = egs.egs_server(8 << 30, max_inflight=2, tile=256, band=2)
    egs.egs_set_allocator(None, None)   # the server keeps the hooks it was created with
    fids = [srv.add_field(np.ascontiguousarray(f.locations().reshape(-1)), f.e(), f.n) for f in fields]
    tickets = [srv.submit(fid, (1.0, 0.1, 0.5), "fp32") for fid in fids]
    got = [srv.wait(t)[0] for t in tickets]
    srv.close()
    assert got == ref
    allocs = sum(1 for c in pool.calls if c[0] == "alloc")
    assert allocs == 2 * len(fields) + len(tickets)
    assert allocs == sum(1 for c in pool.calls if c[0] == "free")
    assert not pool.live

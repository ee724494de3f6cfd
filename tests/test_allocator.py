"""The caller-supplied allocator hook (egs_set_allocator), host side: both
hooks or neither, and a hook that cannot allocate turns into EGS_ERR_OOM
before any device work, after being asked for exactly the evaluation's
workspace (egs_loglik_workspace_bytes).  No GPU is needed: the call fails at
its allocation."""
import numpy as np
import pytest


@pytest.fixture()
def egs():
    import paper_1708_02835_gb300 as m
    m.load_library()
    yield m
    m.egs_set_allocator(None, None)


def test_one_hook_alone_is_rejected(egs):
    with pytest.raises(egs.EgsError) as e:
        egs.egs_set_allocator(lambda n, s: 0, None)
    assert e.value.status == egs.EGS_ERR_ARG
    with pytest.raises(egs.EgsError):
        egs.egs_set_allocator(None, lambda p, n, s: None)
    egs.egs_set_allocator(None, None)
    assert egs.egs_last_error() == ""


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_failing_hook_gives_oom_for_the_workspace_size(egs, prec):
    asked, freed = [], []
    egs.egs_set_allocator(lambda n, s: asked.append(n) or 0, lambda p, n, s: freed.append(p))
    n = 3000
    locs = np.random.default_rng(0).random(2 * n)
    z = np.zeros(n)
    with pytest.raises(egs.EgsError) as e:
        egs.egs_loglik_ex(locs, z, (1.0, 0.1, 0.5), n, prec, tile=256, band=2)
    assert e.value.status == egs.EGS_ERR_OOM
    assert asked == [egs.egs_loglik_workspace_bytes(n, 256, prec, 2)]
    assert freed == []

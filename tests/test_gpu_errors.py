"""Error paths of the boundary, driven from the host without any GPU fault: an allocator that
fails (GSIS_E_OOM, and everything allocated before the failure given back), initial states
with a non-finite or non-positive density or temperature (GSIS_E_INVALID on the host,
GSIS_E_DIVERGED where only the device's moment check can see it)."""
import numpy as np
import pytest

from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GSIS_E_INVALID, GSIS_E_OOM, GSIS_E_DIVERGED = -1, -2, -4


@pytest.mark.parametrize("fail_at", [1, 5, 20])
def test_failing_allocator_gives_oom_and_frees_everything(fail_at):
    import torch

    live, calls = {}, [0]
    dev = torch.cuda.current_device()

    def alloc(nbytes, stream, ctx):
        calls[0] += 1
        if calls[0] >= fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), dev)
        live[p] = nbytes
        return p

    def free(ptr, stream, ctx):
        live.pop(int(ptr))
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = gsis.ALLOC_FN(alloc), gsis.FREE_FN(free)
    p = wl.cavity(n=8, nv=8, Kn=0.1)
    with pytest.raises(gsis.GsisError) as e:
        gsis.Solver(p, precision="f32", torch_memory=False, alloc=a, free=f)
    assert e.value.code == GSIS_E_OOM
    assert calls[0] == fail_at and not live


@pytest.mark.parametrize("field,value", [(0, float("nan")), (0, -0.5), (4, 0.0)])
def test_bad_initial_state_is_refused_on_the_host(field, value):
    """rho and T must be positive: refused before any device work (GSIS_E_INVALID)."""
    p = wl.cavity(n=8, nv=8, Kn=0.1)
    W = p.W0.copy()
    W[13, field] = value
    with pytest.raises(gsis.GsisError) as e:
        gsis.Solver(p, precision="f64", init_W=W, kinetic_presteps=0)
    assert e.value.code == GSIS_E_INVALID, str(e.value)


def test_state_the_device_finds_non_positive_is_reported_as_diverged():
    """An infinite temperature passes the host's check but gives a zero Maxwellian, so the
    device's moment check finds a zero density: GSIS_E_DIVERGED.  A VDF with a non-finite value
    loaded by gsis_set_f is caught the same way."""
    p = wl.cavity(n=8, nv=8, Kn=0.1)
    W = p.W0.copy()
    W[13, 4] = float("inf")
    with pytest.raises(gsis.GsisError) as e:
        gsis.Solver(p, precision="f64", init_W=W, kinetic_presteps=0)
    assert e.value.code == GSIS_E_DIVERGED, str(e.value)
    s = gsis.Solver(p, precision="f32", kinetic_presteps=0)
    f = s.get_f()
    f[21, 5] = float("nan")
    with pytest.raises(gsis.GsisError) as e:
        s.set_f(f)
    assert e.value.code == GSIS_E_DIVERGED, str(e.value)
    s.close()

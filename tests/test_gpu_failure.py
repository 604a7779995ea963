"""Failure detection on the GPU without a fault: each bounded device wait is made to run out (an
arrival that never comes), the kernel raises the time-out status the host reads, and the
context stays usable (a solver steps and matches the oracle afterwards)."""
import pytest

from gpu_common import pair, scaled_close
from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [0, 1], ids=["grid-barrier", "mbarrier"])
def test_bounded_wait_times_out_and_context_survives(which):
    assert gsis.selftest_wait_timeout(which) == gsis.GSIS_E_TIMEOUT
    p = wl.couette(n_cells=12, nv=12, Kn=0.1)
    g, o = pair(p, "f64", "gsis", macro_steps=40)
    g.step()
    o.step()
    scaled_close(g.W(), o.W(), 1e-10, "W after the self-test")

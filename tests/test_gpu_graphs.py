"""Outer steps as captured CUDA graphs (gsis_options.capture_graphs) against direct launches:
the same kernels with the same arguments, so states, residuals and inner step counts agree
exactly, on a rectilinear cavity (cooperative synthetic solve) and on a cylinder O-grid (one
launch per phase of the synthetic solve), in both modes; and after gsis_set_f, which drops the
graphs, and while profiling, which launches directly."""
import numpy as np
import pytest

from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _pair(p, **kw):
    return [gsis.Solver(p, capture_graphs=g, **kw) for g in (1, 0)]


def _why(s):
    return gsis.load().gsis_last_error(s.h).decode()


def _same(a, b, what):
    assert np.array_equal(a.W(), b.W()), what
    assert a.stats() == b.stats(), what


@pytest.mark.parametrize("case", ["cavity_gsis_f32", "cavity_gsis_f64", "cylinder_gsis_f64", "cylinder_dvm_f32"])
def test_graph_steps_equal_direct_launches(case):
    if case.startswith("cavity"):
        p = wl.cavity(n=16, nv=12, Kn=0.1)
        kw = dict(mode="gsis", precision=case[-3:])
    else:
        p = wl.cylinder(n_r=6, n_theta=12, nv=12, R=0.5, R_out=3.0, first=0.15, Ma=0.5, Kn=0.2)
        kw = dict(mode=case.split("_")[1], precision=case[-3:], n_sweeps=2, macro_steps=40)
    g, d = _pair(p, **kw)
    for it in range(5):
        assert g.step() == d.step(), f"{case} eps, step {it}"
        _same(g, d, f"{case}, step {it}")
    # one per mode and state buffer: the kinetic presteps at creation run in DVM mode
    assert g.graphs() == (4 if kw["mode"] == "gsis" else 2), _why(g)
    g.close()
    d.close()


def test_set_f_drops_the_graphs_and_profiling_launches_directly():
    p = wl.cylinder(n_r=6, n_theta=12, nv=12, R=0.5, R_out=3.0, first=0.15, Ma=0.5, Kn=0.2)
    g, d = _pair(p, mode="gsis", precision="f64", n_sweeps=2, macro_steps=40)
    for _ in range(3):
        g.step()
        d.step()
    assert g.graphs() == 4, _why(g)   # presteps (DVM) and GSIS, two state buffers each
    f0, _ = wl.random_vdf(p, seed=3, amp=0.1, W=wl.perturbed_state(p, seed=4, amp=0.02))
    g.set_f(f0)
    d.set_f(f0)
    assert g.graphs() == 0
    for it in range(3):
        assert g.step() == d.step()
        _same(g, d, f"after set_f, step {it}")
    assert g.graphs() == 2
    g.profile(True, reset=True)
    d.profile(True, reset=True)
    n = g.graphs()
    for it in range(2):
        assert g.step() == d.step()
        _same(g, d, f"profiling, step {it}")
    assert g.graphs() == n
    assert g.profile(False)[1] == 2
    g.close()
    d.close()

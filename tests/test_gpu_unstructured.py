"""Unstructured meshes on the GPU against the oracle: tetrahedra, a hybrid prism/hexahedron
cavity (node-sharing least-squares stencils, greedy colour sweeps) and the unstructured forms of
a cavity and a cylinder O-grid (face stencils, GSIS).  FP64 within 1e-10 (rounding order only),
FP32 within the FP32 bounds of the structured tests (2e-5; heat flux 2e-4)."""
import numpy as np
import pytest

from gpu_common import scaled_close
from oracle.oracle import Oracle
from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _pair(p, precision, mode, sweeps, **kw):
    g = gsis.Solver(p, precision=precision, mode=mode, kinetic_presteps=0, n_sweeps=sweeps, macro_tol=0.0, **kw)
    o = Oracle(p, mode=0 if mode == "gsis" else 1, n_sweeps=sweeps, macro_tol=0.0, **kw)
    return g, o


@pytest.mark.parametrize("precision,rel", [("f64", 1e-11), ("f32", 2e-5)])
def test_tetrahedra_kinetic_step_elementwise(precision, rel):
    p = wl.tet_box(n=3, nv=8, Kn=0.2, wall_speed=0.3)
    W = wl.perturbed_state(p, seed=5, amp=0.04)
    g, o = _pair(p, precision, "dvm", 2)
    f0, _ = wl.random_vdf(p, seed=6, amp=0.2, W=W)
    g.set_f(f0)
    o.set_f(f0)
    for it in range(2):
        g.step()
        o.step()
    fg, fo = g.get_f(), o.get_f()[0]
    scale = np.maximum(np.abs(fo).max(axis=0), 1e-3 * np.abs(fo).max())
    assert (np.abs(fg - fo) / scale).max() < rel
    cg, sg, rg, flg = g.wall()
    co, so, ro, flo = o.wall()
    assert np.array_equal(cg, co) and np.array_equal(sg, so)
    np.testing.assert_allclose(rg, ro, rtol=100 * rel)
    g.close()


@pytest.mark.parametrize("precision,rel,relq", [("f64", 1e-10, 1e-10), ("f32", 2e-5, 2e-4)])
def test_hybrid_prism_hexahedron_cavity_kinetic_iteration(precision, rel, relq):
    p = wl.unstructured_cavity(n=6, nv=12, Kn=0.3, lid=0.3, hybrid=0.5)
    g, o = _pair(p, precision, "dvm", 3)
    live = [0, 1, 2, 4, 5, 6, 7, 8, 9]
    for it in range(3):
        g.step()
        o.step()
        hg, ho = g.half_moments(), o.half_moments()
        scaled_close(hg[:, live], ho[:, live], rel, f"{precision} hybrid cavity moments, step {it}")
        scaled_close(hg[:, 12:14], ho[:, 12:14], relq, f"{precision} hybrid cavity heat flux, step {it}", vector=True)
    g.close()


@pytest.mark.parametrize("make", ["cavity", "cylinder"])
def test_unstructured_hexahedra_gsis_steps(make):
    if make == "cavity":
        p = wl.as_unstructured(wl.cavity(n=8, nv=12, Kn=0.2, lid=0.3))
    else:
        p = wl.as_unstructured(wl.cylinder(n_r=5, n_theta=10, nv=12, R=0.5, R_out=3.0, Ma=0.5, Kn=0.2))
    g, o = _pair(p, "f64", "gsis", 2, macro_steps=40)
    for it in range(3):
        g.step()
        o.step()
        scaled_close(g.W()[:, [0, 1, 2, 4]], o.W()[:, [0, 1, 2, 4]], 1e-10, f"{make} unstructured GSIS W, step {it}")
    assert g.stats()[1] == o.macro_iters
    g.close()

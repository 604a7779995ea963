"""Unstructured meshes on the GPU against the oracle: tetrahedra, a hybrid prism/hexahedron
cavity (node-sharing least-squares stencils, greedy colour sweeps, both modes) and the
unstructured forms of a cavity and a cylinder O-grid (face stencils, GSIS).  FP64 within 1e-10 (rounding order only),
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


@pytest.mark.parametrize("make", ["hybrid", "tetrahedra"])
@pytest.mark.parametrize("precision,rel", [("f64", 1e-10), ("f32", 5e-5)])
def test_gsis_steps_on_simplices(make, precision, rel):
    """GSIS outer steps on prisms and tetrahedra (the synthetic solve's gradients over the
    node-sharing stencils, LU-SGS over the greedy colours) from a perturbed state."""
    if make == "hybrid":
        p = wl.unstructured_cavity(n=6, nv=12, Kn=0.2, lid=0.3, hybrid=0.5)
    else:
        p = wl.tet_box(n=3, nv=8, Kn=0.2, wall_speed=0.3)
    W = wl.perturbed_state(p, seed=7, amp=0.03)
    g = gsis.Solver(p, precision=precision, mode="gsis", init_W=W, kinetic_presteps=0, n_sweeps=2, macro_steps=40,
                    macro_tol=0.0)
    o = Oracle(p, W0=W, mode=0, n_sweeps=2, macro_steps=40, macro_tol=0.0)
    for it in range(3):
        g.step()
        o.step()
        scaled_close(g.W()[:, [0, 1, 2, 4]], o.W()[:, [0, 1, 2, 4]], rel, f"{precision} {make} GSIS W, step {it}")
    assert g.stats()[1] == o.macro_iters
    g.close()


def test_gsis_converges_on_a_hybrid_cavity():
    """The hybrid cavity (16^2 squares, half of them split into triangles) at Kn 0.2, where the
    synthetic solve needs the jump term of its viscous face gradients, 40 GSIS steps on the GPU in
    FP64 (eps reaches its rounding floor of 1e-10 .. 1e-9 after about 30): the oracle's converged
    state within 1e-7 of scale."""
    p = wl.unstructured_cavity(n=16, nv=16, Kn=0.2, lid=0.3, hybrid=0.5)
    g = gsis.Solver(p, precision="f64", mode="gsis", kinetic_presteps=0, n_sweeps=4)
    o = Oracle(p, mode=0, n_sweeps=4, nthreads=8)
    eps = []
    for s in (g, o):
        for _ in range(40):
            e = s.step()
        eps.append(e)
    Wg, Wo = g.W(), o.W()
    g.close()
    assert max(eps) < 5e-9
    scaled_close(Wg[:, [0, 1, 2, 4]], Wo[:, [0, 1, 2, 4]], 1e-7, "converged hybrid cavity GSIS W")


def test_rykov_gsis_steps_on_prisms_fp64():
    """The diatomic Rykov gas (two reduced VDFs, the rotational energy equation in the synthetic
    solve) in GSIS on the hybrid prism/hexahedron cavity, with the viscous jump term."""
    p = wl.as_rykov(wl.unstructured_cavity(n=6, nv=10, Kn=0.2, lid=0.3, hybrid=0.5))
    W = wl.perturbed_state(p, seed=8, amp=0.03)
    g = gsis.Solver(p, precision="f64", mode="gsis", init_W=W, kinetic_presteps=0, n_sweeps=2, macro_steps=40,
                    macro_tol=0.0)
    o = Oracle(p, W0=W, mode=0, n_sweeps=2, macro_steps=40, macro_tol=0.0)
    for it in range(2):
        g.step()
        o.step()
        scaled_close(g.W()[:, [0, 1, 2, 4, 5]], o.W()[:, [0, 1, 2, 4, 5]], 1e-10, f"Rykov prism GSIS W, step {it}")
    g.close()

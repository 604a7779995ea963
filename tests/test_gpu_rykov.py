"""Rykov model (diatomic, two reduced VDFs f0, f1; Section 2.2) on the GPU against the FP64
oracle.  FP64: per-iteration moments, states and every VDF value within 1e-10 (rounding order
only).  FP32: per-step states within the FP32 bound of the Shakhov tests (2e-5 of scale)."""
import numpy as np
import pytest

from gpu_common import pair, scaled_close
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _rykov_couette():
    p = wl.as_rykov(wl.couette(n_cells=16, nv=16, Kn=0.1))
    W = p.W0.copy()
    W[:, 5] = 1.15  # rotational temperature out of equilibrium with the translational one
    return p, W


@pytest.mark.parametrize("mode", ["gsis", "dvm"])
def test_rykov_couette_fp64_per_iteration(mode):
    p, W = _rykov_couette()
    g, o = pair(p, "f64", mode, W0=W, macro_steps=100)
    for it in range(4):
        eg = g.step()
        eo = o.step()
        scaled_close(g.half_moments(), o.half_moments(), 1e-10, f"half moments, step {it}")
        scaled_close(g.W(), o.W(), 1e-10, f"W, step {it}")
        assert eg == pytest.approx(eo, rel=1e-8, abs=1e-14)


def test_rykov_random_vdf_one_step_elementwise():
    p = wl.as_rykov(wl.cavity(n=6, nv=12, Kn=0.3, lid=0.3))
    W = wl.perturbed_state(p, seed=7, amp=0.05)
    f0, _ = wl.random_vdf(p, seed=8, amp=0.2, W=W)
    f1 = f0 * (p.d_r * W[:, 5:6] / 4.0) * (1.0 + 0.1 * np.random.default_rng(9).uniform(-1, 1, f0.shape))
    g, o = pair(p, "f64", "dvm")
    g.set_f(f0, f1)
    o.set_f(f0, f1)
    scaled_close(g.half_moments(), o.half_moments(), 1e-12, "moments of set_f")
    g.step()
    o.step()
    gf0, gf1 = g.get_f(both=True)
    of0, of1 = o.get_f()
    scaled_close(gf0, of0, 1e-11, "f0 after one step", vector=True)
    scaled_close(gf1, of1, 1e-11, "f1 after one step", vector=True)
    scaled_close(g.half_moments(), o.half_moments(), 1e-11, "moments after one step")
    # the kinetic wall fluxes, internal energy included
    cg, sg, rg, fg = g.wall()
    co, so, ro, fo = o.wall()
    ig = np.lexsort((sg, cg))
    io = np.lexsort((so, co))
    scaled_close(fg[ig], fo[io], 1e-11, "wall fluxes", vector=True)


def test_rykov_cavity_fp64_gsis_steps():
    p = wl.as_rykov(wl.cavity(n=8, nv=12, Kn=0.2, lid=0.2))
    W = wl.perturbed_state(p, seed=11, amp=0.04)
    g, o = pair(p, "f64", "gsis", W0=W, macro_steps=60)
    for it in range(3):
        g.step()
        o.step()
        scaled_close(g.W(), o.W(), 1e-10, f"W, step {it}")
        scaled_close(g.hot(), o.hot(), 1e-9, f"HoT, step {it}", vector=True)


def test_rykov_couette_fp32_per_iteration():
    """Density and temperatures per column; the velocity as a vector (u_x is zero by symmetry,
    so its own scale would be FP32 noise)."""
    p, W = _rykov_couette()
    g, o = pair(p, "f32", "gsis", W0=W, macro_steps=100)
    for it in range(3):
        g.step()
        o.step()
        Wg, Wo = g.W(), o.W()
        scaled_close(Wg[:, [0, 4, 5]], Wo[:, [0, 4, 5]], 2e-5, f"rho, Tt, Tr, step {it}")
        scaled_close(Wg[:, 1:4], Wo[:, 1:4], 2e-5, f"u, step {it}", vector=True)


def _rel_l2(a, b):
    return np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


@pytest.mark.parametrize("precision,bound", [("f64", 1e-8), ("f32", 1e-4), ("bf16", 1e-3)])
def test_rykov_cavity_converged_matches_oracle(precision, bound):
    """Converged Rykov cavity (uniform cells, so rel-L2 needs no volume weights): the north
    star's bounds for FP32 (1e-4) and BF16 (1e-3) storage; FP64 to 1e-8."""
    p = wl.as_rykov(wl.cavity(n=16, nv=16, Kn=0.1, lid=0.2))
    from paper_2310_18916_gb300 import gsis
    from oracle.oracle import Oracle
    g = gsis.Solver(p, precision=precision, mode="gsis")
    tol = {"f64": 1e-9, "f32": 1e-5, "bf16": 1e-4}[precision]
    done, eps, ok = g.iterate(150, tol)
    o = Oracle(p, mode=0)
    o.presteps(10)
    ho = o.run(150, 1e-9 if precision == "f64" else 1e-6)
    Wg, Wo = g.W(), o.W()
    for k, name in ((0, "rho"), (4, "Tt"), (5, "Tr")):
        e = _rel_l2(Wg[:, k], Wo[:, k])
        assert e < bound, f"{precision} {name}: rel-L2 {e:.2e} after {done} steps (eps {eps:.1e})"

"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

FP64 path: per-iteration moments and states within 1e-10 of the oracle (the differences are
rounding order only).  FP32 path: the VDF is stored in FP32 (unit round-off 6e-8) and the
kinetic arithmetic uses __expf (relative error ~1e-6 near the Maxwellian peak), so per-step
moments agree to a few 1e-6 of their scale; the bound used is 2e-5.  The heat flux is a
cancelling moment: sum |w c^2 c f| / max |q| is about 80 on these cases, so FP32 accumulation
(round-off ~1.5e-6 after the 32-lane tree) leaves ~1.2e-4 of its scale; its bound is 2e-4.
"""
import numpy as np
import pytest

from gpu_common import pair, scaled_close
from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["gsis", "dvm"])
def test_couette_fp64_per_iteration(mode):
    p = wl.couette(n_cells=20, nv=16, Kn=0.1)
    g, o = pair(p, "f64", mode)
    for it in range(4):
        eg = g.step()
        eo = o.step()
        scaled_close(g.half_moments(), o.half_moments(), 1e-10, f"half moments, step {it}")
        scaled_close(g.W(), o.W(), 1e-10, f"W, step {it}")
        assert eg == pytest.approx(eo, rel=1e-8, abs=1e-14)


def test_cavity_fp64_random_vdf_one_step_elementwise():
    """A non-equilibrium start exercises the heat-flux term, limiter, walls and sweeps; every
    f value after one kinetic step must match."""
    p = wl.cavity(n=7, nv=12, Kn=0.3, lid=0.3)
    W = wl.perturbed_state(p, seed=3, amp=0.05)
    f0, _ = wl.random_vdf(p, seed=4, amp=0.2, W=W)
    g, o = pair(p, "f64", "dvm")
    g.set_f(f0)
    o.set_f(f0)
    scaled_close(g.W(), o.W(), 1e-12, "state from set_f")
    g.step()
    o.step()
    fg, fo = g.get_f(), o.get_f()[0]
    assert np.abs(fg - fo).max() <= 1e-12 * np.abs(fo).max()
    cg, sg, rg, flg = g.wall()
    co, so, ro, flo = o.wall()
    ig, io = np.lexsort((cg, sg)), np.lexsort((co, so))     # the two number wall faces differently
    assert np.array_equal(cg[ig], co[io]) and np.array_equal(sg[ig], so[io])
    np.testing.assert_allclose(rg[ig], ro[io], rtol=1e-12)
    scaled_close(flg[ig], flo[io], 1e-11, "wall flux")
    # per cell sum of the outward kinetic face fluxes (the oracle keeps them face by face)
    scaled_close(g.kinetic_flux_sum()[:, :5], o.face_flux().sum(axis=1)[:, :5], 1e-10, "kinetic flux sum")


def test_cavity_fp64_gsis_steps_from_random_vdf():
    p = wl.cavity(n=9, nv=12, Kn=0.1, lid=0.2)
    f0, _ = wl.random_vdf(p, seed=7, amp=0.1)
    g, o = pair(p, "f64", "gsis", macro_steps=60)
    g.set_f(f0)
    o.set_f(f0)
    for it in range(3):
        g.step()
        o.step()
        scaled_close(g.half_moments(), o.half_moments(), 1e-10, f"half moments, step {it}")
        scaled_close(g.W(), o.W(), 1e-10, f"W, step {it}")
    scaled_close(g.get_f(), o.get_f()[0], 1e-10, "f after 3 steps")


@pytest.mark.parametrize("mode", ["gsis", "dvm"])
def test_cavity_fp32_per_iteration(mode):
    p = wl.cavity(n=12, nv=16, Kn=0.1)
    g, o = pair(p, "f32", mode, macro_steps=100)
    for it in range(3):
        g.step()
        o.step()
        hg, ho = g.half_moments(), o.half_moments()
        scaled_close(hg[:, :12], ho[:, :12], 2e-5, f"half moments, step {it}")
        scaled_close(hg[:, 12:15], ho[:, 12:15], 2e-4, f"heat flux, step {it}", vector=True)
        scaled_close(g.W(), o.W(), 2e-5, f"W, step {it}")


def test_wall_loads_match_oracle_wall_fluxes():
    """a10: force, energy flux and the drag / heat-flux coefficients on chosen walls, from the
    kinetic wall fluxes of the last step, against the same sums of the oracle's per-face wall
    fluxes (FP64 path, three GSIS steps)."""
    p = wl.cavity(n=12, nv=16, Kn=0.1, lid=0.16)
    g, o = pair(p, "f64", "gsis", macro_steps=50)
    for _ in range(3):
        g.step()
        o.step()
    _, side, _, fl = o.wall()
    rho, U, A = 1.0, 0.16, 1.0
    for sides, d in (([3], (1.0, 0.0, 0.0)), ([0, 1, 2, 3], (0.0, 1.0, 0.0)), ([2], (0.6, 0.8, 0.0))):
        sel = np.isin(side, sides)
        F = fl[sel, 1:4].sum(axis=0)
        Q = fl[sel, 4].sum()
        ref = np.array([F[0], F[1], F[2], Q, F @ np.array(d) / (0.5 * rho * U ** 2 * A), Q / (0.5 * rho * U ** 3 * A)])
        out = g.wall_loads(sides, d, rho, U, A)
        fs = np.abs(F).max()
        scale = np.array([fs, fs, fs, max(abs(Q), fs * U), fs / (0.5 * rho * U ** 2 * A),
                          max(abs(Q), fs * U) / (0.5 * rho * U ** 3 * A)])
        err = np.abs(out - ref) / scale
        assert err.max() < 1e-10, f"sides {sides}: {err}"
    with pytest.raises(gsis.GsisError):
        g.wall_loads([3], (1.0, 0.0, 0.0), 0.0, U, A)

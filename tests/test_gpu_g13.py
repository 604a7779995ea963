"""The Grad-13 wall flux of the synthetic solve (Section 3.3, Eqs. G13_VDF and GSIS-DVM-flux,
wall_flux = GSIS_WALL_G13) on the GPU against the oracle with the same option: GSIS outer steps
on the rectilinear cavity (Shakhov and Rykov, FP64 and FP32 storage) and on the cylinder O-grid
(the general synthetic solve), W within the bounds of the Maxwellian-flux tests."""
import numpy as np
import pytest

from gpu_common import scaled_close
from oracle.oracle import Oracle
from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
G13 = 1


def _pair(p, precision, steps, **opts):
    g = gsis.Solver(p, precision=precision, mode="gsis", kinetic_presteps=0, macro_tol=0.0, wall_flux=G13, **opts)
    o = Oracle(p, mode=0, macro_tol=0.0, wall_flux=G13, **opts)
    out = []
    for _ in range(steps):
        g.step()
        o.step()
        out.append((g.W(), o.W()))
    g.close()
    return out


@pytest.mark.parametrize("rykov", [False, True])
def test_cavity_gsis_steps_with_the_grad13_wall_flux_fp64(rykov):
    p = wl.cavity(n=10, nv=12, Kn=0.1, lid=0.3)
    if rykov:
        p = wl.as_rykov(p)
    for it, (Wg, Wo) in enumerate(_pair(p, "f64", 3)):
        scaled_close(Wg, Wo, 1e-10, f"G13 cavity W, step {it}")


def test_cavity_gsis_steps_with_the_grad13_wall_flux_fp32():
    p = wl.cavity(n=10, nv=16, Kn=0.1, lid=0.3)
    for it, (Wg, Wo) in enumerate(_pair(p, "f32", 2)):
        scaled_close(Wg[:, [0, 1, 2, 4]], Wo[:, [0, 1, 2, 4]], 2e-5, f"G13 FP32 cavity W, step {it}")


def test_cylinder_gsis_steps_with_the_grad13_wall_flux_fp64():
    p = wl.cylinder(n_r=6, n_theta=12, nv=12, R=0.5, R_out=3.0, Ma=0.5, Kn=0.2)
    for it, (Wg, Wo) in enumerate(_pair(p, "f64", 2, n_sweeps=2)):
        scaled_close(Wg, Wo, 1e-10, f"G13 cylinder W, step {it}")

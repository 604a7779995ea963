"""Parity at the benchmark's sizes and launch configurations, through the C ABI.

- The 128^2 x 32^3 cavity (537M points) in FP32 storage, the configuration the benchmark's
  FP32 form times (the shared-memory colour ring, 32^3 tiled velocity blocks): one complete GSIS
  outer step against the FP64 oracle run on every host core, every cell's half-step moments and
  W within the FP32 bounds of the small-case tests (2e-5; heat flux 2e-4 of its scale).
- The same workload in FP64, one GSIS outer step, every cell within 1e-10.
- The sphere O-grid of the body benchmark (32 x 24 x 48 cells, radial ratio 1.1), with 12^3
  uniform velocities, FP32: one kinetic step with two colour passes and the benchmark's
  pseudo-time step, every f value against the oracle.
"""
import os

import numpy as np
import pytest

from gpu_common import scaled_close
from oracle.oracle import Oracle
from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
CORES = os.cpu_count() or 1


@pytest.fixture(scope="module")
def cavity_oracle_step():
    """One GSIS outer step of the oracle on the 128^2 x 32^3 cavity (all host cores)."""
    p = wl.cavity(n=128, nv=32, Kn=0.1, lid=0.16)
    o = Oracle(p, mode=0, nthreads=CORES, macro_tol=0.0)
    o.step()
    out = (p, o.half_moments(), o.W())
    del o
    return out


@pytest.mark.parametrize("precision,rel,relq", [("f32", 2e-5, 2e-4), ("f64", 1e-10, 1e-10)])
def test_benchmark_cavity_one_gsis_step_cell_by_cell(cavity_oracle_step, precision, rel, relq):
    p, Mo, Wo = cavity_oracle_step
    g = gsis.Solver(p, precision=precision, mode="gsis", kinetic_presteps=0, macro_tol=0.0)
    g.step()
    Mg, Wg = g.half_moments(), g.W()
    g.close()
    scaled_close(Mg[:, :12], Mo[:, :12], rel, f"{precision} 128^2 x 32^3 half-step moments")
    scaled_close(Mg[:, 12:15], Mo[:, 12:15], relq, f"{precision} 128^2 x 32^3 heat flux", vector=True)
    scaled_close(Wg, Wo, rel, f"{precision} 128^2 x 32^3 W after the synthetic solve")


def test_sphere_benchmark_mesh_fp32_kinetic_step_elementwise():
    p = wl.sphere(n_r=32, n_pol=24, n_az=48, nv=12, R=0.5, R_out=5.0, first=0.0224, Ma=4.0, Kn=0.05, vmax=12.0)
    opts = dict(n_sweeps=2, kin_inv_dt=1000.0, kinetic_presteps=0)
    g = gsis.Solver(p, precision="f32", mode="dvm", **opts)
    g.step()
    fg = g.get_f()
    Mg = g.half_moments()
    g.close()
    o = Oracle(p, mode=1, n_sweeps=2, kin_inv_dt=1000.0, nthreads=CORES)
    o.step()
    fo = o.get_f()[0]
    # FP32 storage of f and FP32 exponentials: a few 1e-6 of each velocity's scale for the
    # velocities that carry the moments; velocities in the Maxwellians' tails, below 1e-3 of the
    # peak, against that floor (there the FP32 exponential's relative error grows with its
    # argument)
    scale = np.maximum(np.abs(fo).max(axis=0), 1e-3 * np.abs(fo).max())
    err = (np.abs(fg - fo) / scale).max()
    assert err < 2e-5, f"sphere 32x24x48 x 12^3: f after one kinetic step differs by {err:.3e} of its scale"
    scaled_close(Mg[:, :12], o.half_moments()[:, :12], 2e-5, "sphere half-step moments")

"""Edge cases of the GPU path against the FP64 oracle: a 3D box (three active axes), odd
velocity counts (a xi = 0 node on every axis, ragged octants padded with weight-0 slots),
rectangular grids, the rest state, colour rings in device scratch (bit-identical to shared memory;
3D boxes too large for it against the oracle), and one kinetic step of
the full benchmark workload (128^2 cells x 32^3 velocities) compared cell by cell."""
import os

import numpy as np
import pytest

from gpu_common import pair, scaled_close
from oracle.oracle import Oracle
from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_box3d_fp64_random_vdf_step_and_gsis_steps():
    p = wl.box3d(ni=5, nj=4, nk=3, nv=10, Kn=0.2, wall_speed=0.25)
    W = wl.perturbed_state(p, seed=21, amp=0.04)
    f0, _ = wl.random_vdf(p, seed=22, amp=0.2, W=W)
    g, o = pair(p, "f64", "dvm")
    g.set_f(f0)
    o.set_f(f0)
    g.step()
    o.step()
    scaled_close(g.get_f(), o.get_f()[0], 1e-11, "f after one step", vector=True)
    scaled_close(g.half_moments(), o.half_moments(), 1e-11, "moments after one step")
    g2, o2 = pair(p, "f64", "gsis", W0=W, macro_steps=60)
    for it in range(3):
        g2.step()
        o2.step()
        scaled_close(g2.W(), o2.W(), 1e-10, f"box W, step {it}")


@pytest.mark.parametrize("nv", [11, 15])
def test_odd_velocity_counts_fp64(nv):
    """Odd counts put a node at xi = 0 (no transport along that axis) and make the octants'
    velocity counts ragged (not multiples of 32)."""
    p = wl.couette(n_cells=12, nv=nv, Kn=0.1)
    g, o = pair(p, "f64", "gsis", macro_steps=80)
    for it in range(3):
        g.step()
        o.step()
        scaled_close(g.half_moments(), o.half_moments(), 1e-10, f"nv={nv} moments, step {it}")


def test_rectangular_cavity_fp64():
    p = wl.cavity(n=9, ny=5, nv=12, Kn=0.15, lid=0.2)
    g, o = pair(p, "f64", "gsis", macro_steps=60)
    for it in range(3):
        g.step()
        o.step()
        scaled_close(g.W(), o.W(), 1e-10, f"9x5 cavity W, step {it}")


def test_rest_state_stays_at_rest():
    """Walls at rest at the gas temperature: the gas stays uniform and at rest.  (On a midpoint
    velocity grid the Maxwellian's discrete temperature differs from 1 by the quadrature error,
    so the first steps move the uniform state to the discrete equilibrium: eps falls, but the
    field never becomes non-uniform.)"""
    p = wl.cavity(n=12, nv=16, Kn=0.1, lid=0.0)
    g, o = pair(p, "f64", "gsis", macro_steps=100)
    for _ in range(6):
        g.step()
        o.step()
    W = g.W()
    scaled_close(W[:, [0, 4]], o.W()[:, [0, 4]], 1e-10, "rest state rho, T")
    assert np.abs(W[:, 0] - W[:, 0].mean()).max() < 1e-8
    assert np.abs(W[:, 1:4]).max() < 1e-8
    assert np.abs(W[:, 4] - W[:, 4].mean()).max() < 1e-8
    assert abs(W[:, 4].mean() - 1.0) < 1e-5
    # (eps itself is not small here: the velocity is round-off, ~1e-10, above eps's zero-field
    # threshold, and its relative change is of order one)


@pytest.mark.parametrize("precision,rykov", [("f32", False), ("bf16", False), ("f64", True)])
def test_global_ring_is_bit_identical(precision, rykov):
    """kinetic_ring = 1 keeps the sweep's colour ring and wall face values in device scratch
    instead of shared memory. The arithmetic and its order are the same, so the VDF after GSIS
    steps is bit-identical to the shared-memory kernel's."""
    p = wl.box3d(ni=6, nj=5, nk=4, nv=10, Kn=0.2, wall_speed=0.25)
    if rykov:
        p = wl.as_rykov(p)
    W = wl.perturbed_state(p, seed=31, amp=0.04)
    runs = []
    for ring in (0, 1):
        g = gsis.Solver(p, precision=precision, mode="gsis", init_W=W, kinetic_presteps=2, macro_steps=40,
                        kinetic_ring=ring)
        for _ in range(2):
            g.step()
        runs.append((g.get_f(), g.W()))
        g.close()
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))


@pytest.mark.parametrize("precision,n,rel", [("f64", 16, 1e-10), ("f32", 18, 2e-5)])
def test_box3d_beyond_shared_memory(precision, n, rel):
    """A 3D box whose largest colour does not fit in shared memory (16^3 cells in FP64, 18^3 in
    FP32): the ring moves to device scratch by itself, and GSIS steps match the oracle."""
    p = wl.box3d(ni=n, nj=n, nk=n, nv=8, Kn=0.2, wall_speed=0.25)
    assert gsis.footprint_bytes(p, precision) == gsis.footprint_bytes(p, precision, kinetic_ring=1)
    W = wl.perturbed_state(p, seed=33, amp=0.04)
    g, o = pair(p, precision, "gsis", W0=W, macro_steps=60)
    for it in range(2):
        g.step()
        o.step()
        scaled_close(g.W(), o.W(), rel, f"{n}^3 box W, step {it}")


def test_benchmark_workload_one_kinetic_step_cell_by_cell():
    """The full benchmark workload (128^2 x 32^3 = 537M points) in FP64: after one plain kinetic
    step (the kinetic kernels the benchmark times, at its launch configuration) every cell's
    moments match the oracle's."""
    p = wl.cavity(n=128, nv=32, Kn=0.1, lid=0.16)
    g = gsis.Solver(p, precision="f64", mode="dvm", kinetic_presteps=0)
    g.step()
    Mg = g.half_moments()
    g.close()
    o = Oracle(p, mode=1, nthreads=os.cpu_count() or 1)
    o.step()
    scaled_close(Mg, o.half_moments(), 1e-10, "128^2 x 32^3 moments after one step")

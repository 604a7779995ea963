"""Drag and heat-flux coefficients of a sphere in supersonic flow (Ma 1.5, Kn 0.1, diffuse wall
at the free-stream temperature) from converged GSIS solutions on the GPU in FP64, FP32 and BF16
storage, against the FP64 oracle's converged solution on the same inputs: C_D and C_H within
0.5 %.  The mesh is a spherical O-grid with poles and a closed azimuth, the velocity grid is
clustered about the free-stream velocity (the stretched grid of the sphere configuration,
scaled down)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
MA, KN, R = 1.5, 0.1, 0.5


def _problem():
    p = wl.sphere(n_r=8, n_pol=6, n_az=12, nv=4, R=R, R_out=4.0, first=0.08, Ma=MA, Kn=KN)
    return wl.with_clustered_velocities(p, 20, 8.0)


def _coefficients(force, energy, U):
    q = 0.5 * 1.0 * U ** 2 * np.pi * R ** 2
    return force[0] / q, energy / (q * U)


@pytest.fixture(scope="module")
def oracle_converged():
    p = _problem()
    o = Oracle(p, mode=0, n_sweeps=2)
    o.presteps(10)
    for _ in range(80):
        if o.step() < 1e-6:
            break
    assert o.eps < 1e-6
    cell, side, rw, fl = o.wall()
    U = float(np.linalg.norm(p.wall_u[1]))
    return _coefficients(fl[:, 1:4].sum(0), fl[:, 4].sum(), U)


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16"])
def test_sphere_drag_and_heat_flux_match_the_oracle(oracle_converged, precision):
    p = _problem()
    U = float(np.linalg.norm(p.wall_u[1]))
    s = gsis.Solver(p, precision=precision, mode="gsis", n_sweeps=2)
    best, since = np.inf, 0
    for _ in range(100):
        e = s.step()
        best, since = (e, 0) if e < best else (best, since + 1)
        if e < 1e-6 or since >= 15:
            break
    out = s.wall_loads([0], (1.0, 0.0, 0.0), 1.0, U, np.pi * R ** 2)
    s.close()
    cd, ch = oracle_converged
    assert cd > 0 and ch > 0
    assert abs(out[4] / cd - 1) < 5e-3, f"{precision}: C_D {out[4]:.6f} vs oracle {cd:.6f}"
    assert abs(out[5] / ch - 1) < 5e-3, f"{precision}: C_H {out[5]:.6f} vs oracle {ch:.6f}"


def _continued(make_solver, steps_max=80):
    """Mach continuation 1.5 -> 2.0 -> 2.5: each stage starts from the previous converged state
    (its Maxwellian) with the faster free stream, 10 kinetic presteps, then GSIS to eps < 1e-6."""
    W = None
    for Ma in (1.5, 2.0, 2.5):
        p = wl.with_clustered_velocities(
            wl.sphere(n_r=8, n_pol=6, n_az=12, nv=4, R=R, R_out=4.0, first=0.08, Ma=Ma, Kn=KN), 20, 8.0)
        W, loads = make_solver(p, W, steps_max)
    return p, W, loads


def test_sphere_at_mach_2_5_by_continuation_matches_the_oracle():
    """A converged supersonic body-fitted case above Ma 2: the sphere at Ma 2.5 (Kn 0.1), reached
    by Mach continuation from the Ma-1.5 solution (an impulsive Ma-2.5 start loses positivity
    next to the rear pole).  GPU in FP64 and FP32 storage against the oracle's own continuation:
    C_D and C_H within 0.5 %, the wake's lowest density within 1 %."""
    def oracle_stage(p, W, n):
        o = Oracle(p, W0=W, mode=0, n_sweeps=2)
        o.presteps(10)
        for _ in range(n):
            if o.step() < 1e-6:
                break
        assert o.eps < 1e-6
        _, _, _, fl = o.wall()
        U = float(np.linalg.norm(p.wall_u[1]))
        return o.W(), _coefficients(fl[:, 1:4].sum(0), fl[:, 4].sum(), U)

    p, Wo, (cd, ch) = _continued(oracle_stage)
    assert cd > 0 and ch > 0 and Wo[:, 0].min() < 0.2

    for precision in ("f64", "f32"):
        def gpu_stage(q, W, n):
            s = gsis.Solver(q, precision=precision, mode="gsis", n_sweeps=2, init_W=W)
            best, since = np.inf, 0
            for _ in range(n):
                e = s.step()
                best, since = (e, 0) if e < best else (best, since + 1)
                if e < 1e-6 or since >= 15:
                    break
            U = float(np.linalg.norm(q.wall_u[1]))
            out = s.wall_loads([0], (1.0, 0.0, 0.0), 1.0, U, np.pi * R ** 2)
            Wg = s.W()
            s.close()
            return Wg, (out[4], out[5])

        _, Wg, (cdg, chg) = _continued(gpu_stage)
        assert abs(cdg / cd - 1) < 5e-3, f"{precision}: C_D {cdg:.6f} vs oracle {cd:.6f}"
        assert abs(chg / ch - 1) < 5e-3, f"{precision}: C_H {chg:.6f} vs oracle {ch:.6f}"
        assert abs(Wg[:, 0].min() / Wo[:, 0].min() - 1) < 1e-2

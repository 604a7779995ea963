"""Positive face values (gsis_options.positive_faces) on body-fitted grids, against the oracle
with the same option: the kinetic steps element by element (FP64) and within the FP32 bound, and
the sphere at Ma 4 reached by Mach continuation 1.5 -> 2.5 -> 3.25 -> 4 (which the linear
reconstruction cannot pass beyond about Ma 2.75: the wake next to the rear pole empties),
C_D and C_H within 0.5 % of the oracle's."""
import numpy as np
import pytest

from gpu_common import scaled_close
from oracle.oracle import Oracle
from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
R, KN = 0.5, 0.1


def _sphere(Ma):
    p = wl.sphere(n_r=8, n_pol=6, n_az=12, nv=4, R=R, R_out=4.0, first=0.08, Ma=Ma, Kn=KN)
    return wl.with_clustered_velocities(p, 20, 8.0)


@pytest.mark.parametrize("precision,rel", [("f64", 1e-11), ("f32", 2e-5)])
def test_kinetic_steps_with_positive_faces(precision, rel):
    """Three DVM steps (1/dt = 1000) from the impulsive Ma-4 start on the sphere, where the
    linear reconstruction undershoots in the wake: every f value in FP64, W in FP32."""
    p = _sphere(4.0)
    opts = dict(n_sweeps=2, kin_inv_dt=1000.0)
    g = gsis.Solver(p, precision=precision, mode="dvm", kinetic_presteps=0, positive_faces=1, **opts)
    o = Oracle(p, mode=1, positive_faces=1, **opts)
    for it in range(3):
        g.step()
        o.step()
        scaled_close(g.W(), o.W(), rel, f"{precision} positive faces W, step {it}")
    if precision == "f64":
        fg, fo = g.get_f(), o.get_f()[0]
        assert np.abs(fg - fo).max() <= 1e-11 * np.abs(fo).max()
    g.close()


def _continuation(stage):
    W, out = None, None
    for Ma in (1.5, 2.5, 3.25, 4.0):
        W, out = stage(_sphere(Ma), W)
    return W, out


def _coefficients(fl, U):
    q = 0.5 * U ** 2 * np.pi * R ** 2
    return fl[:, 1].sum() / q, fl[:, 4].sum() / (q * U)


def test_sphere_at_mach_4_by_continuation_with_positive_faces():
    def oracle_stage(p, W):
        o = Oracle(p, W0=W, mode=0, n_sweeps=2, positive_faces=1)
        o.presteps(10)
        for _ in range(60):
            if o.step() < 1e-6:
                break
        assert o.eps < 1e-6
        _, _, _, fl = o.wall()
        return o.W(), _coefficients(fl, float(np.linalg.norm(p.wall_u[1])))

    Wo, (cd, ch) = _continuation(oracle_stage)
    assert cd > 0 and ch > 0 and Wo[:, 0].min() > 0.02

    for precision in ("f64", "f32"):
        def gpu_stage(p, W):
            s = gsis.Solver(p, precision=precision, mode="gsis", n_sweeps=2, init_W=W, positive_faces=1)
            best, since = np.inf, 0
            for _ in range(60):
                e = s.step()
                best, since = (e, 0) if e < best else (best, since + 1)
                if e < 1e-6 or since >= 15:
                    break
            U = float(np.linalg.norm(p.wall_u[1]))
            out = s.wall_loads([0], (1.0, 0.0, 0.0), 1.0, U, np.pi * R ** 2)
            Wg = s.W()
            s.close()
            return Wg, (out[4], out[5])

        Wg, (cdg, chg) = _continuation(gpu_stage)
        assert abs(cdg / cd - 1) < 5e-3, f"{precision}: C_D {cdg:.6f} vs oracle {cd:.6f}"
        assert abs(chg / ch - 1) < 5e-3, f"{precision}: C_H {chg:.6f} vs oracle {ch:.6f}"
        assert abs(Wg[:, 0].min() / Wo[:, 0].min() - 1) < 1e-2

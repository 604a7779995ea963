"""General (curvilinear) structured meshes on the GPU against the FP64 oracle: the kinetic
iteration and GSIS on a cylinder O-grid (wall inside, far field outside, wrapped azimuth) and a
sphere O-grid (pole sides of zero area), with several colour passes per step; FP64 element by
element, FP32 within its rounding; the Rykov model; wall fluxes and loads; the collisionless
reservoir slab against its exact discrete solution."""
import numpy as np
import pytest

from gpu_common import scaled_close
from oracle.oracle import Oracle
from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def run_pair(p, precision, steps, n_sweeps, W0=None, f0=None):
    g = gsis.Solver(p, precision=precision, mode="dvm", init_W=W0, kinetic_presteps=0, n_sweeps=n_sweeps)
    o = Oracle(p, W0=W0, mode=1, n_sweeps=n_sweeps)
    if f0 is not None:
        g.set_f(f0)
        o.set_f(f0)
    out = []
    for _ in range(steps):
        g.step()
        o.step()
        out.append((g.W(), o.W()))
    return g, o, out


def wall_match(g, o, rel):
    cg, sg, rg, flg = g.wall()
    co, so, ro, flo = o.wall()
    assert np.array_equal(cg, co) and np.array_equal(sg, so)
    np.testing.assert_allclose(rg, ro, rtol=rel)
    scaled_close(flg, flo, rel * 10, "wall flux")


@pytest.mark.parametrize("n_sweeps", [1, 3])
def test_cylinder_ogrid_fp64(n_sweeps):
    p = wl.cylinder(n_r=6, n_theta=12, nv=12, R=0.5, R_out=3.0, first=0.15, Ma=0.5, Kn=0.2, T_w=1.5)
    W = wl.perturbed_state(p, seed=41, amp=0.04)
    f0, _ = wl.random_vdf(p, seed=42, amp=0.2, W=W)
    g, o, out = run_pair(p, "f64", 3, n_sweeps, W0=W, f0=f0)
    for it, (Wg, Wo) in enumerate(out):
        scaled_close(Wg, Wo, 1e-11, f"cylinder W, step {it}")
    fg, fo = g.get_f(), o.get_f()[0]
    assert np.abs(fg - fo).max() <= 1e-11 * np.abs(fo).max()
    wall_match(g, o, 1e-11)


def test_sphere_ogrid_fp64():
    p = wl.sphere(n_r=4, n_pol=5, n_az=8, nv=10, R=0.5, R_out=3.0, Ma=0.6, Kn=0.3)
    W = wl.perturbed_state(p, seed=43, amp=0.04)
    g, o, out = run_pair(p, "f64", 3, 2, W0=W)
    for it, (Wg, Wo) in enumerate(out):
        scaled_close(Wg, Wo, 1e-11, f"sphere W, step {it}")
    fg, fo = g.get_f(), o.get_f()[0]
    assert np.abs(fg - fo).max() <= 1e-11 * np.abs(fo).max()
    wall_match(g, o, 1e-11)


def test_cylinder_rykov_fp64():
    p = wl.as_rykov(wl.cylinder(n_r=5, n_theta=10, nv=10, R=0.5, R_out=3.0, Ma=0.5, Kn=0.2, T_w=1.3))
    W = wl.perturbed_state(p, seed=44, amp=0.04)
    g, o, out = run_pair(p, "f64", 2, 2, W0=W)
    for it, (Wg, Wo) in enumerate(out):
        scaled_close(Wg, Wo, 1e-11, f"Rykov cylinder W, step {it}")
    fg, fo = g.get_f(both=True), o.get_f()
    assert np.abs(fg[0] - fo[0]).max() <= 1e-11 * np.abs(fo[0]).max()
    assert np.abs(fg[1] - fo[1]).max() <= 1e-11 * np.abs(fo[1]).max()


@pytest.mark.parametrize("precision,rel", [("f32", 2e-5), ("bf16", 2e-3)])
def test_cylinder_ogrid_reduced_precision(precision, rel):
    p = wl.cylinder(n_r=6, n_theta=12, nv=16, R=0.5, R_out=3.0, Ma=0.5, Kn=0.2)
    g, o, out = run_pair(p, precision, 3, 2)
    for it, (Wg, Wo) in enumerate(out):
        # rho and temperatures per column, the velocity as one vector (u_z of this 2D flow is
        # rounding noise, which a per-column scale would compare instead of the flow)
        scaled_close(Wg[:, [0, 4, 5]], Wo[:, [0, 4, 5]], rel, f"{precision} cylinder rho, T, step {it}")
        scaled_close(Wg[:, 1:4], Wo[:, 1:4], rel, f"{precision} cylinder u, step {it}", vector=True)


def test_cylinder_pseudo_time_step_fp64():
    """kin_inv_dt > 0 (the delta form with 1/dt on the diagonal) against the oracle."""
    p = wl.cylinder(n_r=6, n_theta=12, nv=12, R=0.5, R_out=3.0, Ma=1.5, Kn=0.1)
    g = gsis.Solver(p, precision="f64", mode="dvm", kinetic_presteps=0, n_sweeps=2, kin_inv_dt=5.0)
    o = Oracle(p, mode=1, n_sweeps=2, kin_inv_dt=5.0)
    for it in range(3):
        g.step()
        o.step()
        scaled_close(g.W(), o.W(), 1e-11, f"cylinder W with 1/dt = 5, step {it}")


def test_cylinder_wall_loads_match_oracle():
    """a10 on a curved body: force and drag coefficient on the cylinder from the wall fluxes."""
    p = wl.cylinder(n_r=6, n_theta=16, nv=12, R=0.5, R_out=3.0, Ma=0.5, Kn=0.3)
    g, o, _ = run_pair(p, "f64", 3, 2)
    _, side, _, fl = o.wall()
    U = p.wall_u[1][0]
    F = fl[side == 0, 1:4].sum(axis=0)
    out = g.wall_loads([0], (1.0, 0.0, 0.0), 1.0, U, 1.0)
    np.testing.assert_allclose(out[:3], F, rtol=1e-10, atol=1e-12 * np.abs(F).max())
    assert out[4] == pytest.approx(F[0] / (0.5 * U * U), rel=1e-10)


def test_reservoir_wall_exact_on_gpu():
    U = (0.0, 0.3, 0.0)
    p = wl.reservoir_wall(n_cells=8, nv=16, U=U, T_inf=1.0, T_w=2.0, Kn=1e9)
    W0 = np.tile([0.5, 0.0, 0.0, 0.0, 1.5, 1.5], (p.ncells, 1))
    g = gsis.Solver(p, precision="f64", mode="dvm", init_W=W0, kinetic_presteps=0)
    for _ in range(4):
        g.step()
    f = g.get_f()
    X, Y, Z = np.meshgrid(p.vx, p.vy, p.vz, indexing="ij")

    def M(rho, u, T):
        return (rho * (np.pi * T) ** -1.5 * np.exp(-((X - u[0]) ** 2 + (Y - u[1]) ** 2 + (Z - u[2]) ** 2) / T)).transpose(2, 1, 0).ravel()

    vx = X.transpose(2, 1, 0).ravel()
    w = np.multiply.outer(np.multiply.outer(p.wx, p.wy), p.wz).transpose(2, 1, 0).ravel()
    Minf, Mw = M(1.0, U, 1.0), M(1.0, (0, 0, 0), 2.0)
    up, dn = vx > 0, vx < 0
    rho_w = (w[up] * vx[up] * Minf[up]).sum() / (w[dn] * -vx[dn] * Mw[dn]).sum()
    exact = np.where(up, Minf, rho_w * Mw)
    assert np.abs(f - exact[None, :]).max() < 1e-6 * np.abs(exact).max()


def gsis_pair(p, precision, n_sweeps, W0=None, macro_steps=40):
    g = gsis.Solver(p, precision=precision, mode="gsis", init_W=W0, kinetic_presteps=0, n_sweeps=n_sweeps,
                    macro_steps=macro_steps, macro_tol=0.0)
    o = Oracle(p, W0=W0, mode=0, n_sweeps=n_sweeps, macro_steps=macro_steps, macro_tol=0.0)
    return g, o


@pytest.mark.parametrize("body", ["cylinder", "sphere"])
def test_gsis_steps_on_ogrids_fp64(body):
    """The synthetic solve on general meshes (Rusanov + NSF faces, far-field faces against the
    free stream, wall faces by the equilibrium wall flux, red/black LU-SGS) after the kinetic
    step, GSIS outer steps against the oracle."""
    if body == "cylinder":
        p = wl.cylinder(n_r=6, n_theta=12, nv=12, R=0.5, R_out=3.0, first=0.15, Ma=0.5, Kn=0.2, T_w=1.5)
    else:
        p = wl.sphere(n_r=4, n_pol=5, n_az=8, nv=10, R=0.5, R_out=3.0, Ma=0.6, Kn=0.3)
    W = wl.perturbed_state(p, seed=45, amp=0.03)
    g, o = gsis_pair(p, "f64", 2, W0=W)
    for it in range(3):
        g.step()
        o.step()
        scaled_close(g.W(), o.W(), 1e-10, f"{body} GSIS W, step {it}")
    assert g.stats()[1] == o.macro_iters
    fg, fo = g.get_f(), o.get_f()[0]
    assert np.abs(fg - fo).max() <= 1e-10 * np.abs(fo).max()


def test_gsis_rykov_cylinder_fp64():
    p = wl.as_rykov(wl.cylinder(n_r=5, n_theta=10, nv=10, R=0.5, R_out=3.0, Ma=0.5, Kn=0.2, T_w=1.3))
    g, o = gsis_pair(p, "f64", 2)
    for it in range(2):
        g.step()
        o.step()
        scaled_close(g.W(), o.W(), 1e-10, f"Rykov cylinder GSIS W, step {it}")


def test_relaxed_gsis_update_on_a_cylinder_fp64():
    """gsis_options.relax = 0.5: the state after each GSIS step is the blend of the half-step
    moments and the synthetic solution, on the GPU as in the oracle, element by element."""
    p = wl.cylinder(n_r=6, n_theta=12, nv=12, R=0.5, R_out=3.0, first=0.15, Ma=0.5, Kn=0.2, T_w=1.5)
    W = wl.perturbed_state(p, seed=46, amp=0.03)
    g = gsis.Solver(p, precision="f64", mode="gsis", init_W=W, kinetic_presteps=0, n_sweeps=2, macro_steps=40,
                    macro_tol=0.0, relax=0.5)
    o = Oracle(p, W0=W, mode=0, n_sweeps=2, macro_steps=40, macro_tol=0.0, relax=0.5)
    for it in range(3):
        g.step()
        o.step()
        scaled_close(g.W(), o.W(), 1e-10, f"relaxed cylinder GSIS W, step {it}")
    g.close()


def test_viscous_jump_weight_on_a_cylinder_fp64():
    """gsis_options.visc_jump = 0.5 on a hexahedral O-grid (where the default is none): the
    synthetic solve's viscous face gradients with the jump term, GSIS steps element by element."""
    p = wl.cylinder(n_r=6, n_theta=12, nv=12, R=0.5, R_out=3.0, first=0.15, Ma=0.5, Kn=0.2, T_w=1.5)
    W = wl.perturbed_state(p, seed=47, amp=0.03)
    g = gsis.Solver(p, precision="f64", mode="gsis", init_W=W, kinetic_presteps=0, n_sweeps=2, macro_steps=40,
                    macro_tol=0.0, visc_jump=0.5)
    o = Oracle(p, W0=W, mode=0, n_sweeps=2, macro_steps=40, macro_tol=0.0, visc_jump=0.5)
    o0 = Oracle(p, W0=W, mode=0, n_sweeps=2, macro_steps=40, macro_tol=0.0)
    for it in range(3):
        g.step()
        o.step()
        o0.step()
        scaled_close(g.W(), o.W(), 1e-10, f"cylinder GSIS W with the jump term, step {it}")
    assert np.abs(o.W() - o0.W()).max() > 1e-8   # the term is there
    g.close()


def test_gsis_cylinder_fp32_and_early_exit():
    p = wl.cylinder(n_r=6, n_theta=12, nv=16, R=0.5, R_out=3.0, Ma=0.5, Kn=0.2)
    g, o = gsis_pair(p, "f32", 2, macro_steps=60)
    for it in range(2):
        g.step()
        o.step()
        scaled_close(g.W(), o.W(), 5e-5, f"FP32 cylinder GSIS W, step {it}")
    # with the inner tolerance the solve stops early, at the oracle's inner step
    g2 = gsis.Solver(p, precision="f64", mode="gsis", kinetic_presteps=0, n_sweeps=2, macro_steps=300,
                     macro_tol=1e-6)
    o2 = Oracle(p, mode=0, n_sweeps=2, macro_steps=300, macro_tol=1e-6)
    g2.step()
    o2.step()
    assert g2.stats()[1] == o2.macro_iters < 300
    scaled_close(g2.W(), o2.W(), 1e-10, "cylinder GSIS W with the inner tolerance")


def test_euler_presteps_then_gsis_on_a_cylinder_fp64():
    """The inviscid presteps at creation (slip wall, far field against the free stream), then
    GSIS steps from the Maxwellian of their result, against the oracle."""
    p = wl.cylinder(n_r=6, n_theta=12, nv=12, R=0.5, R_out=3.0, Ma=0.8, Kn=0.1)
    g = gsis.Solver(p, precision="f64", mode="gsis", kinetic_presteps=0, n_sweeps=2, macro_steps=40, macro_tol=0.0,
                    euler_presteps=60)
    o = Oracle(p, mode=0, n_sweeps=2, macro_steps=40, macro_tol=0.0)
    o.euler_presteps(60)
    scaled_close(g.W(), o.W(), 1e-10, "W after the Euler presteps")
    for it in range(2):
        g.step()
        o.step()
        scaled_close(g.W(), o.W(), 1e-10, f"GSIS W after Euler presteps, step {it}")


def test_free_molecular_cylinder_drag_on_gpu():
    """The GPU's wall loads on the cylinder at Kn = 1e6 against the discrete free-molecular force
    (the closed form of tests/test_oracle_farfield.py), FP64 and FP32."""
    from test_oracle_farfield import cylinder_free_molecular, free_molecular_force

    p = cylinder_free_molecular()
    S = Oracle(p, mode=1).geometry()[2].reshape(32, 10, 6, 3)[:, 0, 0, :]
    exact = free_molecular_force(p, S, p.wall_u[1], p.wall_T[0])
    U = p.wall_u[1][0]
    for precision, rel in (("f64", 1e-4), ("f32", 2e-4)):
        g = gsis.Solver(p, precision=precision, mode="dvm", kinetic_presteps=0, n_sweeps=2, kin_inv_dt=2.0)
        for _ in range(15):
            g.step()
        out = g.wall_loads([0], (1.0, 0.0, 0.0), 1.0, U, 1.0)
        g.close()
        assert abs(out[0] - exact[0]) < rel * exact[0], precision
        assert abs(out[1]) < 1e-6 * exact[0], precision
        assert out[4] == pytest.approx(out[0] / (0.5 * U * U), rel=1e-12)

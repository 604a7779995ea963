"""Pins of the oracle's gas model (Section 2) against what the paper and the mathematics fix."""
import math
import os

import numpy as np
import pytest

from conftest import read_golden
from oracle import oracle as O
from paper_2310_18916_gb300 import workloads as wl


def _gas(model=wl.SHAKHOV, omega=0.81, Kn=0.1, d_r=0.0, Z_r=1.0, A=(2 / 3, 0, 0, 1)):
    p = wl.couette(n_cells=2, nv=4)
    p.model, p.omega, p.Kn, p.d_r, p.Z_r, p.A = model, omega, Kn, d_r, Z_r, tuple(A)
    return p


def test_eucken_factors_match_section5(golden_dir):
    """Eq. mu_kappa with the nitrogen A of Section 5 must give the printed Eucken factors.

    f_t = kappa_t/(c_vt mu) with c_vt = (3/2) R, f_r = kappa_r/(c_vr mu) with c_vr = (d_r/2) R,
    and R = 1/2 in the solver's units (R T -> T/2)."""
    g = read_golden(os.path.join(golden_dir, "eucken_n2.txt"))
    p = _gas(wl.RYKOV, omega=g["omega"], d_r=g["d_r"], Z_r=g["Z_r"], A=g["A"])
    mu = 0.37
    kt, kr = O.conductivity(p, mu)
    R = 0.5
    assert kt / (1.5 * R * mu) == pytest.approx(g["f_t"], abs=1.5e-3)
    assert kr / (g["d_r"] / 2 * R * mu) == pytest.approx(g["f_r"], abs=1.5e-3)


def test_monatomic_conductivity_is_prandtl_two_thirds():
    """Shakhov/monatomic: kappa = 15 mu R / 4 (Pr = c_p mu / kappa = 2/3 with c_p = 5R/2)."""
    p = _gas()
    mu = 0.8
    kt, kr = O.conductivity(p, mu)
    R = 0.5
    assert (2.5 * R) * mu / kt == pytest.approx(2.0 / 3.0, rel=1e-14)
    assert kr == 0.0


def _shakhov_textbook(st, xi, Pr=2.0 / 3.0):
    """Shakhov's model in its usual dimensional form with R = 1/2:
    f_M [1 + (1 - Pr) c.q / (5 p R T) (c^2/(R T) - 5)], f_M = rho (2 pi R T)^{-3/2} exp(-c^2/(2RT))."""
    R = 0.5
    rho, u, T, q = st[0], np.array(st[1:4]), st[4], np.array(st[6:9])
    c = np.asarray(xi) - u
    c2 = c @ c
    p = rho * R * T
    fm = rho * (2 * math.pi * R * T) ** -1.5 * math.exp(-c2 / (2 * R * T))
    return fm * (1 + (1 - Pr) * (c @ q) / (5 * p * R * T) * (c2 / (R * T) - 5))


def test_g0t_is_shakhov_with_prandtl_two_thirds():
    rng = np.random.default_rng(1)
    p = _gas()
    for _ in range(50):
        st = np.zeros(12)
        st[0] = rng.uniform(0.3, 3)
        st[1:4] = rng.uniform(-1, 1, 3)
        st[4] = st[5] = rng.uniform(0.3, 3)
        st[6:9] = rng.uniform(-0.3, 0.3, 3)
        xi = rng.uniform(-3, 3, 3)
        g0, g1 = O.reference(p, st, xi)
        assert g0 == pytest.approx(_shakhov_textbook(st, xi), rel=1e-12, abs=1e-300)
        assert g1 == 0.0


def test_rykov_reduces_to_shakhov_without_internal_modes():
    """d_r = 0 and A_tt = 2/3: q0 = q_t, T = T_t, so g_0r = g_0t and g0 = g_0t for any Z_r."""
    rng = np.random.default_rng(2)
    sh = _gas()
    for Zr in (1.0, 3.5, 50.0):
        ry = _gas(wl.RYKOV, d_r=0.0, Z_r=Zr, A=(2 / 3, 0.0, 0.0, 0.7))
        for _ in range(20):
            st = np.zeros(12)
            st[0] = rng.uniform(0.5, 2)
            st[1:4] = rng.uniform(-1, 1, 3)
            st[4] = rng.uniform(0.5, 2)
            st[5] = rng.uniform(0.5, 2)
            st[6:12] = rng.uniform(-0.2, 0.2, 6)
            xi = rng.uniform(-3, 3, 3)
            assert O.reference(ry, st, xi)[0] == pytest.approx(O.reference(sh, st, xi)[0], rel=1e-12)


def _vgrid(n, vmax=6.0):
    x, w = wl.midpoint_grid(n, -vmax, vmax)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel()
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1), W


def _moments_of_reference(p, st, n):
    xi, w = _vgrid(n)
    g = np.array([O.reference(p, st, x) for x in xi])
    u = st[1:4]
    c = xi - u
    c2 = (c * c).sum(1)
    out = dict(rho=w @ g[:, 0], mom=(w[:, None] * c * g[:, 0:1]).sum(0), e=w @ (0.5 * c2 * g[:, 0]),
               q=(w[:, None] * (0.5 * c2)[:, None] * c * g[:, 0:1]).sum(0), e1=w @ g[:, 1],
               q1=(w[:, None] * c * g[:, 1:2]).sum(0))
    return out


def test_shakhov_collision_conserves_and_relaxes_heat_flux_to_one_third():
    """Moments of g_0t: mass, momentum and energy of the state exactly (up to quadrature),
    heat flux (1 - Pr) q = q/3.  The quadrature error must fall as the grid is refined."""
    p = _gas()
    st = np.array([1.3, 0.2, -0.1, 0.05, 1.1, 1.1, 0.05, -0.08, 0.03, 0, 0, 0])
    errs = []
    for n in (8, 12, 16, 24):
        m = _moments_of_reference(p, st, n)
        err = max(abs(m["rho"] - st[0]) / st[0], np.abs(m["mom"]).max(), abs(m["e"] - 0.75 * st[0] * st[4]),
                  np.abs(m["q"] - st[6:9] / 3).max())
        errs.append(err)
    assert errs[-1] < 1e-10
    assert errs[0] > errs[1] > errs[2]


def test_rykov_collision_conserves_total_energy_and_relaxes_temperatures():
    """Rykov-type model (Section 2.2): moments of g0, g1 conserve mass, momentum and total
    energy; translational/internal energies relax towards T = (3Tt + d_r Tr)/(3 + d_r) at rate
    1/Z_r; heat fluxes relax by the rates A."""
    d_r, Zr, A = 2.0, 3.5, wl.N2_A
    p = _gas(wl.RYKOV, omega=0.74, d_r=d_r, Z_r=Zr, A=A)
    st = np.array([0.9, 0.1, 0.0, -0.2, 1.4, 0.8, 0.03, -0.02, 0.01, -0.01, 0.02, 0.015])
    m = _moments_of_reference(p, st, 24)
    rho, Tt, Tr = st[0], st[4], st[5]
    T = (3 * Tt + d_r * Tr) / (3 + d_r)
    assert m["rho"] == pytest.approx(rho, rel=1e-10)
    assert np.abs(m["mom"]).max() < 1e-10
    # (3/2) rho R T_t -> 3 rho Tt / 4 and (d_r/2) rho R T_r -> d_r rho Tr / 4
    assert m["e"] == pytest.approx(0.75 * rho * ((1 - 1 / Zr) * Tt + T / Zr), rel=1e-10)
    assert m["e1"] == pytest.approx(d_r * rho / 4 * ((1 - 1 / Zr) * Tr + T / Zr), rel=1e-10)
    assert m["e"] + m["e1"] == pytest.approx(0.75 * rho * Tt + d_r * rho * Tr / 4, rel=1e-10)
    # heat fluxes of (g0, g1): (I - A)(q_t, q_r), the homogeneous relaxation d q/dt = -A q / tau
    # that defines A (Section 2.2); the translational flux of g0 is the c^2/2-weighted moment
    Att, Atr, Art, Arr = A
    qt, qr = st[6:9], st[9:12]
    np.testing.assert_allclose(m["q"], qt - (Att * qt + Atr * qr), atol=1e-10)
    np.testing.assert_allclose(m["q1"], qr - (Art * qt + Arr * qr), atol=1e-10)


def test_tau_from_dimensional_definitions():
    """tau = mu(Tt)/p_t with Kn = mu(T0)/(p0 L) sqrt(pi R T0/2), done in SI units for an
    argon-like gas and then scaled by L / v0, v0 = sqrt(2 R T0)."""
    R, T0, p0, L = 208.13, 273.15, 2.0, 0.05
    Kn, omega = 0.07, 0.81
    mu0 = Kn * p0 * L / math.sqrt(math.pi * R * T0 / 2)
    rho0 = p0 / (R * T0)
    v0 = math.sqrt(2 * R * T0)
    p = _gas(Kn=Kn, omega=omega)
    for rho_hat, T_hat in ((1.0, 1.0), (0.4, 2.5), (3.0, 0.3)):
        rho, T = rho_hat * rho0, T_hat * T0
        mu = mu0 * (T / T0) ** omega
        tau = mu / (rho * R * T)
        assert O.tau(p, rho_hat, T_hat) == pytest.approx(tau * v0 / L, rel=1e-12)


def test_venkatakrishnan_special_values():
    """Venkatakrishnan's function with eps = 0: phi = (y^2 + 2y)/(y^2 + y + 2), y = Dm/D2:
    0 at y = 0, 3/4 at y = 1, 1 at y = 2, -> 1 as y -> inf; 1 when D2 = 0; odd symmetry."""
    f = O.venkat_face
    assert f(0.0, 0.3, 0.0) == 0.0
    assert f(0.3, 0.3, 0.0) == pytest.approx(0.75, rel=1e-15)
    assert f(0.6, 0.3, 0.0) == pytest.approx(1.0, rel=1e-15)
    assert f(1e6, 1.0, 0.0) == pytest.approx(1.0, rel=1e-5)
    assert f(0.7, 0.0, 1e-3) == 1.0
    assert f(-0.2, -0.5, 1e-4) == pytest.approx(f(0.2, 0.5, 1e-4), rel=1e-15)
    # eps^2 dominates: phi -> 1
    assert f(1e-6, 1e-6, 1.0) == pytest.approx(1.0, rel=1e-5)


def _one_cell(model, nv=24, vmax=6.0, Kn=0.1):
    """A single periodic cell (no transport): the kinetic step is the homogeneous relaxation."""
    xs = np.array([0.0, 1.0])
    v, w = wl.midpoint_grid(nv, -vmax, vmax)
    p = wl.Problem(ni=1, nj=1, nk=1, nodes=wl.box_nodes(xs, xs, xs), bc=[wl.PERIODIC] * 6,
                   wall_u=np.zeros((6, 3)), wall_T=np.ones(6), vx=v, vy=v.copy(), vz=v.copy(), wx=w,
                   wy=w.copy(), wz=w.copy(), Kn=Kn, W0=np.array([[1.0, 0.0, 0.0, 0.0, 1.0, 1.0]]), name="one_cell")
    if model == wl.RYKOV:
        p.model, p.omega, p.d_r, p.Z_r, p.A = wl.RYKOV, 0.74, 2.0, 5.0, wl.N2_A
    return p


def _nonequilibrium_f(p, seed):
    """Seeded f0, f1 with nonzero translational and internal heat fluxes: Maxwellians of
    (rho, u, Tt) times a positive, smooth, direction-dependent modulation."""
    rng = np.random.default_rng(seed)
    X, Y, Z = np.meshgrid(p.vx, p.vy, p.vz, indexing="ij")
    xi = np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(), Z.transpose(2, 1, 0).ravel()], 1)
    W = (p.wx[None, None, :] * p.wy[None, :, None] * p.wz[:, None, None]).ravel()
    rho, Tt, Tr = 1.1, 0.9, 1.2
    u = np.array([0.1, -0.05, 0.02])
    c = xi - u
    c2 = (c * c).sum(1)
    M = rho * (np.pi * Tt) ** -1.5 * np.exp(-c2 / Tt)
    a, b = rng.uniform(-0.06, 0.06, 3), rng.uniform(-0.06, 0.06, 3)
    f0 = M * (1 + (c @ a) * (c2 / Tt - 2.5) * np.exp(-c2 / (4 * Tt)))
    f1 = p.d_r * Tr / 4 * M * (1 + (c @ b) * np.exp(-c2 / (4 * Tt)))
    return xi, W, f0, f1


def _heat_fluxes(xi, W, f0, f1):
    """q_t = sum w (c^2/2) c f0 and q_r = sum w c f1 about the mean velocity (Eq. getmoment)."""
    rho = W @ f0
    u = (W[:, None] * xi * f0[:, None]).sum(0) / rho
    c = xi - u
    c2 = (c * c).sum(1)
    qt = (W[:, None] * (0.5 * c2)[:, None] * c * f0[:, None]).sum(0)
    qr = (W[:, None] * c * f1[:, None]).sum(0)
    return rho, u, (W @ (0.5 * c2 * f0)) / (0.75 * rho), qt, qr


@pytest.mark.parametrize("inv_dt", [0.0, 3.0])
def test_rykov_heat_fluxes_relax_at_rate_A_over_tau(inv_dt):
    """The 2x2 map that builds q0, q1 (Section 2.2, below Eq. general_model) is fixed by what A
    means: the relaxation rates of the heat fluxes.  In a homogeneous gas Eq. general_model
    gives d(q_t, q_r)/dt = -(1/tau) A (q_t, q_r), so the kinetic step on one periodic cell, whose
    delta form with 1/dt = k reads (k + 1/tau) df = (g - f)/tau, must give
        (q_t, q_r)^{n+1/2} = (I - A / (1 + k tau)) (q_t, q_r)^n.
    The expected values come from A alone (the nitrogen rates of Section 5 with Z_r = 5), never
    from the q0, q1 matrix; swapping A_tr and A_rt inside the oracle's reference distribution,
    or a sign slip in either off-diagonal entry, fails this test."""
    p = _one_cell(wl.RYKOV)
    xi, W, f0, f1 = _nonequilibrium_f(p, seed=7)
    rho, u, Tt, qt, qr = _heat_fluxes(xi, W, f0, f1)
    assert min(np.abs(qt).max(), np.abs(qr).max()) > 1e-3
    o = O.Oracle(p, mode=1, kin_inv_dt=inv_dt, nthreads=1)
    o.set_f(f0[None, :], f1[None, :])
    o.step()
    m = o.half_moments()[0]
    delta = 1.0 / (1.0 + inv_dt * O.tau(p, rho, Tt))
    Att, Atr, Art, Arr = p.A
    want_t = qt - delta * (Att * qt + Atr * qr)
    want_r = qr - delta * (Art * qt + Arr * qr)
    scale = max(np.abs(qt).max(), np.abs(qr).max())
    np.testing.assert_allclose(m[12:15], want_t, atol=1e-9 * scale)
    np.testing.assert_allclose(m[15:18], want_r, atol=1e-9 * scale)


def test_shakhov_heat_flux_relaxes_at_two_thirds_over_tau():
    """Shakhov (Pr = 2/3, A_tt = 2/3): the heat flux of the homogeneous step is q (1 - (2/3) delta)."""
    p = _one_cell(wl.SHAKHOV)
    xi, W, f0, _ = _nonequilibrium_f(p, seed=8)
    rho, u, Tt, qt, _ = _heat_fluxes(xi, W, f0, np.zeros_like(f0))
    o = O.Oracle(p, mode=1, kin_inv_dt=2.0, nthreads=1)
    o.set_f(f0[None, :])
    o.step()
    delta = 1.0 / (1.0 + 2.0 * O.tau(p, rho, Tt))
    np.testing.assert_allclose(o.half_moments()[0][12:15], qt * (1 - 2.0 / 3.0 * delta), atol=1e-9 * np.abs(qt).max())

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
    1/Z_r; heat fluxes follow the 2x2 relaxation map."""
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
    Att, Atr, Art, Arr = A
    qt, qr = st[6:9], st[9:12]
    q0 = ((2 - 3 * Att) * Zr + 1) * qt - 3 * Atr * Zr * qr
    q1 = -Art * Zr * qt + (-Arr * Zr + 1) * qr
    np.testing.assert_allclose(m["q"], ((1 - 1 / Zr) * qt + q0 / Zr) / 3, atol=1e-10)
    np.testing.assert_allclose(m["q1"], (1 - 1 / Zr) * qr + q1 / Zr, atol=1e-10)


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

"""Pins of the oracle's Grad-13 wall flux (Section 3.3, Eqs. G13_VDF and GSIS-DVM-flux).

The oracle takes the half-range moments of the 13-moment VDF in closed form.  Here the VDF is
built independently: its stress and heat-flux coefficients are solved for on a velocity grid so
that its moments are the given sigma, q_t (and q_r), and the half-range fluxes are then taken by
quadrature in the face's frame (Gauss-Legendre along the normal on the half that moves into the
wall, midpoint rules across).  A slip in the closed form (a dropped tangential moment, a wrong
sign of u_n, a swapped sigma component) fails the comparison; with sigma = q = 0 the flux is the
Maxwellian one."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2310_18916_gb300 import workloads as wl

RHO, U, T, TR = 1.3, np.array([0.4, -0.2, 0.1]), 1.2, 1.1
N = np.array([0.6, 0.64, -0.48])
SIG = np.array([0.05, -0.02, -0.03, 0.015, -0.01, 0.02])   # xx yy zz xy xz yz (traceless)
QT = np.array([0.03, -0.02, 0.04])
QR = np.array([0.01, 0.02, -0.015])
TW = 0.8


def _oracle(rykov):
    p = wl.cavity(n=2, nv=4, Kn=0.1)
    uw = np.cross(N, [0.0, 0.0, 1.0])
    uw = 0.3 * uw / np.linalg.norm(uw)       # a wall moving in its own plane
    p.wall_u[0], p.wall_T[0] = uw, TW
    if rykov:
        p = wl.as_rykov(p)
    return Oracle(p, mode=1, nthreads=1), p, uw


def _frame(n):
    t1 = np.cross(n, [1.0, 0.0, 0.0])
    t1 /= np.linalg.norm(t1)
    return np.stack([n, t1, np.cross(n, t1)])     # rows: n, t1, t2


def _sigma(s):
    return np.array([[s[0], s[3], s[4]], [s[3], s[1], s[5]], [s[4], s[5], s[2]]])


def _grad13(rho, u, T, sig, qt, qr, d_r, Tr):
    """The 13-moment VDF pair as functions of peculiar velocity c (n, 3): coefficients of
    c_i c_j (symmetric traceless) and of c_i (c^2/T - 5/2) fitted on a full-space grid so
    that sigma_ij = int c_i c_j f0 - p delta_ij and q_t = int c^2 c f0 / 2; for f1 the
    coefficient of c_i M so that int c f1 = q_r, on top of (d_r T_r / 4) f0."""
    x = (np.arange(48) + 0.5) / 48 * 16 - 8
    h = x[1] - x[0]
    c = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3) * np.sqrt(T)
    w = (h * np.sqrt(T)) ** 3
    M = rho * (np.pi * T) ** -1.5 * np.exp(-(c * c).sum(1) / T)
    c2 = (c * c).sum(1)
    pairs = [(0, 0), (1, 1), (0, 1), (0, 2), (1, 2)]      # zz = -(xx + yy)
    cols = []
    for a, b in pairs:
        if a == b:
            cols.append(c[:, a] ** 2 - c[:, 2] ** 2)
        else:
            cols.append(2 * c[:, a] * c[:, b])
    for a in range(3):
        cols.append(c[:, a] * (c2 / T - 2.5))
    basis = np.stack(cols, 1)
    # moments of M * basis: stress (6) and heat flux (3) rows
    p = rho * T / 2
    rows = []
    for a, b in [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]:
        rows.append(w * (M * c[:, a] * c[:, b]) @ basis)
    for a in range(3):
        rows.append(w * (M * 0.5 * c2 * c[:, a]) @ basis)
    rhs = np.concatenate([[sig[0], sig[1], sig[2], sig[3], sig[4], sig[5]], qt])
    coef = np.linalg.lstsq(np.array(rows), rhs, rcond=None)[0]
    assert np.allclose(np.array(rows) @ coef, rhs, atol=1e-12)
    # f1's heat-flux coefficient
    k = np.array([w * (M * c[:, a] * c[:, a]) .sum() for a in range(3)])
    gam = qr / k

    def f0(cc):
        cc2 = (cc * cc).sum(1)
        Mc = rho * (np.pi * T) ** -1.5 * np.exp(-cc2 / T)
        b = []
        for a, bb in pairs:
            b.append(cc[:, a] ** 2 - cc[:, 2] ** 2 if a == bb else 2 * cc[:, a] * cc[:, bb])
        for a in range(3):
            b.append(cc[:, a] * (cc2 / T - 2.5))
        return Mc * (1 + np.stack(b, 1) @ coef), Mc

    def f1(cc):
        g0, Mc = f0(cc)
        return d_r * Tr / 4 * g0 + Mc * (cc @ gam)

    return f0, f1


def _half_range_flux(rho, u, T, sig, qt, qr, rykov, d_r, Tr, uw, Tw):
    f0, f1 = _grad13(rho, u, T, sig, qt, qr, d_r, Tr)
    R = _frame(N)
    # xi = xn n + y t1 + z t2, xn > 0 (into the wall) for the gas, xn < 0 for the wall
    gx, gw = np.polynomial.legendre.leggauss(64)
    smax = np.sqrt(max(T, Tw)) * 9 + 3
    xn = (gx + 1) / 2 * smax
    wn = gw / 2 * smax
    y = (np.arange(64) + 0.5) / 64 * 2 * smax - smax
    wy = 2 * smax / 64
    XN, Y, Z = np.meshgrid(xn, y, y, indexing="ij")
    W3 = (wn[:, None, None] * wy * wy) * np.ones_like(XN)
    xi_in = XN.reshape(-1, 1) * R[0] + Y.reshape(-1, 1) * R[1] + Z.reshape(-1, 1) * R[2]
    w = W3.reshape(-1)
    g0 = f0(xi_in - u)[0]
    g1 = f1(xi_in - u) if rykov else np.zeros_like(g0)
    xin = XN.reshape(-1)
    F = np.zeros(6)
    F[0] = (w * xin * g0).sum()
    F[1:4] = (w * xin * g0) @ xi_in
    F[4] = (w * xin * (0.5 * (xi_in * xi_in).sum(1) * g0 + g1)).sum()
    F[5] = (w * xin * g1).sum()
    # the wall's half: rho_w M(u_w, T_w) with zero net mass flux
    xi_out = -XN.reshape(-1, 1) * R[0] + Y.reshape(-1, 1) * R[1] + Z.reshape(-1, 1) * R[2]
    cw = xi_out - uw
    Mw = (np.pi * Tw) ** -1.5 * np.exp(-(cw * cw).sum(1) / Tw)
    xo = -XN.reshape(-1)
    m_out = (w * xo * Mw).sum()
    rw = -F[0] / m_out
    F[0] += rw * m_out
    F[1:4] += rw * (w * xo * Mw) @ xi_out
    e1w = d_r * Tw / 4 * Mw if rykov else 0 * Mw
    F[4] += rw * (w * xo * (0.5 * (xi_out * xi_out).sum(1) * Mw + e1w)).sum()
    F[5] += rw * (w * xo * e1w).sum()
    return F


@pytest.mark.parametrize("rykov", [False, True])
def test_grad13_wall_flux_matches_quadrature_of_the_13_moment_vdf(rykov):
    o, p, uw = _oracle(rykov)
    pr = np.concatenate([[RHO], U, [T, TR if rykov else T]])
    m18 = np.zeros(18)
    m18[6:12], m18[12:15] = SIG, QT
    if rykov:
        m18[15:18] = QR
    got = o.wall_flux(1, 0, pr, m18, N)
    ref = _half_range_flux(RHO, U, T, SIG, QT, QR if rykov else 0 * QR, rykov, p.d_r, TR if rykov else T, uw, TW)
    scale = np.abs(ref).max()
    assert np.abs(got[:5] - ref[:5]).max() < 1e-9 * scale, (got, ref)
    if rykov:
        assert abs(got[5] - ref[5]) < 1e-9 * scale
    # the Grad-13 terms matter: the flux differs from the Maxwellian one
    eq = o.wall_flux(0, 0, pr, m18, N)
    assert np.abs(got[:5] - eq[:5]).max() > 1e-3 * scale


@pytest.mark.parametrize("rykov", [False, True])
def test_grad13_wall_flux_without_stress_or_heat_flux_is_the_maxwellian_flux(rykov):
    o, p, uw = _oracle(rykov)
    for un in (-0.7, 0.0, 0.35, 1.4):
        u = U + (un - U @ N) * N
        pr = np.concatenate([[RHO], u, [T, TR if rykov else T]])
        m18 = np.zeros(18)
        g = o.wall_flux(1, 0, pr, m18, N)
        e = o.wall_flux(0, 0, pr, m18, N)
        np.testing.assert_allclose(g, e, rtol=1e-12, atol=1e-14)
        assert abs(g[0]) < 1e-13   # zero net mass flux through the wall


def test_grad13_and_maxwellian_wall_fluxes_share_the_fixed_point():
    """Both wall models enter the synthetic solve as increments on the kinetic wall flux, so GSIS
    converges to the same state with either (and, on this cavity, in the same number of outer
    steps: the increment form already carries the kinetic wall flux).  The closed cavity's mass
    rescaling ties its fixed point to the synthetic solve at the 1e-6 level (1e-6 here on 10^2
    cells, 2e-11 on 16^2), hence the bound."""
    out = {}
    for wf in (0, 1):
        p = wl.cavity(n=10, nv=12, Kn=0.1, lid=0.16)
        o = Oracle(p, mode=0, wall_flux=wf)
        for it in range(60):
            if o.step() < 1e-9:
                break
        out[wf] = (o.W(), it)
    W0, W1 = out[0][0], out[1][0]
    scale = np.maximum(np.abs(W0).max(axis=0), 1e-3 * np.abs(W0).max())
    assert (np.abs(W1 - W0) / scale).max() < 1e-5
    assert abs(out[0][1] - out[1][1]) <= 1

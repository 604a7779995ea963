"""Pins of the oracle's finite-volume geometry, LSQ gradient and limiter."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2310_18916_gb300 import workloads as wl


def _skewed(ni=5, nj=4, nk=3):
    """A box mapped by a constant shear (determinant 1): every cell is the same parallelepiped."""
    p = wl.box3d(ni, nj, nk, nv=4)
    X = p.nodes.copy()
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    p.nodes = np.ascontiguousarray(np.stack([x + 0.3 * y + 0.1 * z, y + 0.2 * z, z], -1))
    J = np.array([[1, 0.3, 0.1], [0, 1, 0.2], [0, 0, 1]])
    return p, J


def test_rectilinear_volumes_and_closed_faces():
    p = wl.cavity(n=6, nv=4, stretch=1.5)
    o = Oracle(p, mode=1)
    vol, xc, S, xf = o.geometry()
    xs = p.nodes[0, 0, :, 0]
    dz = p.nodes[1, 0, 0, 2] - p.nodes[0, 0, 0, 2]
    expect = np.outer(np.diff(xs), np.diff(xs)).ravel() * dz   # cells ordered i fastest (j outer)
    np.testing.assert_allclose(vol, expect, rtol=1e-13)
    assert vol.sum() == pytest.approx(1.0 * 1.0 * dz, rel=1e-13)


def test_skewed_geometry_parallelepiped():
    p, J = _skewed()
    o = Oracle(p, mode=1)
    vol, xc, S, xf = o.geometry()
    h = np.array([1 / 5, 0.8 / 4, 0.6 / 3])
    np.testing.assert_allclose(vol, np.linalg.det(J) * h.prod(), rtol=1e-12)
    # geometric conservation: the closed surface of every cell sums to zero
    assert np.abs(S.sum(axis=1)).max() < 1e-15
    # outward: S . (x_f - x_c) > 0 on every face
    assert ((S * (xf - xc[:, None, :])).sum(-1) > 0).all()
    # face area vector of an x-face = (e_y x e_z) of the mapped cell
    ey, ez = J[:, 1] * h[1], J[:, 2] * h[2]
    np.testing.assert_allclose(S[0, 1], np.cross(ey, ez), rtol=1e-12)


def test_lsq_gradient_exact_for_linear_fields_on_skewed_mesh():
    p, J = _skewed()
    o = Oracle(p, mode=1)
    _, xc, _, _ = o.geometry()
    a = np.array([0.7, -1.3, 2.1])
    q = 0.4 + xc @ a
    for c in range(o.nc):
        np.testing.assert_allclose(o.cell_gradient(c, q), a, rtol=1e-10, atol=1e-12)


def test_limiter_is_one_for_linear_data_and_small_at_extrema():
    p = wl.cavity(n=8, nv=4)
    o = Oracle(p, mode=1)
    _, xc, _, _ = o.geometry()
    q = 1.0 + 0.5 * xc[:, 0] - 0.2 * xc[:, 1]
    interior = [i + 8 * j for i in range(1, 7) for j in range(1, 7)]
    for c in interior:
        assert o.cell_limiter(c, q) == pytest.approx(1.0, abs=1e-12)
    # a strict local maximum with a non-zero LSQ slope (east neighbour higher than the west):
    # no face value may exceed the maximum, so the limiter nearly switches the slope off
    q = np.zeros(o.nc)
    q[27], q[28], q[26] = 1.0, 0.5, 0.0
    g = o.cell_gradient(27, q)
    assert g[0] == pytest.approx(0.25 * 8, rel=1e-13)   # (q_E - q_W) / (2 dx), dx = 1/8
    # east face: D2 = g dx/2 = 1/8, Dm = 0; eps^2 = (K h)^3 with h = V^(1/3) = 1/8 (K = 1):
    # phi = eps^2 / (2 D2^2 + eps^2) = (1/512) / (1/32 + 1/512) = 1/17
    assert o.cell_limiter(27, q) == pytest.approx(1.0 / 17.0, rel=1e-12)


def test_body_grid_generators():
    """The O-grid inputs: geometric radial spacing with the requested first width and the
    configuration-3 ratio, a closed azimuth (the last node row is the first), exact poles."""
    r = wl.radial_nodes(32, 0.5, 5.0, first=0.0224)
    d = np.diff(r)
    assert r[0] == 0.5 and r[-1] == 5.0 and abs(d[0] - 0.0224) < 1e-12
    np.testing.assert_allclose(d[1:-1] / d[:-2], d[1] / d[0], rtol=1e-9)
    assert abs(d[1] / d[0] - 1.1) < 1e-3
    c = wl.cylinder(n_r=4, n_theta=6, nv=4)
    assert np.array_equal(c.nodes[:, -1], c.nodes[:, 0])
    s = wl.sphere(n_r=3, n_pol=4, n_az=6, nv=4)
    assert np.array_equal(s.nodes[-1], s.nodes[0])                                # closed azimuth
    for pole in (0, -1):  # every azimuth meets at one point on the axis
        pts = s.nodes[:, pole, :, :]
        assert np.abs(pts[..., 1:]).max() == 0.0
        assert np.abs(pts - pts[:1]).max() == 0.0


def test_capsule_mesh_converges_to_the_body_of_revolution():
    """The capsule O-grid (heat-shield cap of radius 1 up to the shoulder 60 degrees off the axis,
    then a 33-degree cone closing on the axis): the fluid volume and the wetted area of the wall
    faces approach the closed forms of the body (spherical segment + cone) as the polar and
    azimuthal resolution double: the volume at second order, the area (the shoulder's kink falls
    between nodes at a different place on each mesh) at better than order 1.4 over the range."""
    a, beta = np.pi / 3, np.radians(33.0)
    h, rs = 1 - np.cos(a), np.sin(a)
    slant = rs / np.sin(beta)
    V_body = np.pi * h * h * (3 - h) / 3 + np.pi * rs * rs * (slant * np.cos(beta)) / 3
    A_body = 2 * np.pi * h + np.pi * rs * slant
    R_out = 3.0
    V_exact = 4 / 3 * np.pi * R_out ** 3 - V_body
    ev, ea = [], []
    for k in (1, 2, 4, 8):
        p = wl.capsule(n_r=3, n_pol=6 * k, n_az=8 * k, nv=4, R_out=R_out)
        vol, _, S, _ = Oracle(p, mode=1, nthreads=4).geometry()
        ev.append(abs(vol.sum() / V_exact - 1))
        wall = np.arange(p.ncells) % p.ni == 0
        ea.append(abs(np.linalg.norm(S[wall, 0], axis=1).sum() / A_body - 1))
    assert all(x > y for x, y in zip(ev, ev[1:])) and all(x > y for x, y in zip(ea, ea[1:]))
    assert ev[-1] < 3e-3 and ea[-1] < 5e-3
    assert ev[0] / ev[1] > 3.5 and ev[1] / ev[2] > 3.5 and ev[2] / ev[3] > 3.5
    assert ea[0] / ea[-1] > 8 ** 1.4
    assert p.model == wl.RYKOV and abs(p.Ma - 10.0) < 1e-12


def test_positive_faces_keep_a_steep_fall_positive_and_second_order_where_smooth():
    """orc_opts.positive_faces: where the linear face value falls below the cell value (d < 0)
    the face takes q_i^2 / (q_i - d).  On a steep monotone fall into zero the Venkatakrishnan-
    limited linear value undershoots to below zero (its eps^2 term lets it); the option keeps
    it positive and leaves the rising face untouched.  On smooth positive data the two forms
    differ by d^2 / (q_i - d): a quarter as much when the mesh spacing halves (3.7 and 3.9 from
    16^2 to 64^2 cells, the limiter still slightly below 1)."""
    p = wl.cavity(n=8, nv=4)
    lin, pos = Oracle(p, mode=1), Oracle(p, mode=1, positive_faces=1)
    q = np.zeros(lin.nc)
    q[26], q[27], q[28] = 1.0, 0.05, 0.0            # west, cell, east along x
    fl, fp = lin.cell_faces(27, q), pos.cell_faces(27, q)
    phi, g = lin.cell_limiter(27, q), lin.cell_gradient(27, q)
    d_east = phi * g[0] / 16                          # r = dx / 2 = 1/16 towards the east face
    assert d_east < 0 and fl[1] == pytest.approx(0.05 + d_east, rel=1e-12) and fl[1] < 0
    assert fp[1] > 0 and fp[1] == pytest.approx(0.05 ** 2 / (0.05 - d_east), rel=1e-12)
    assert fp[0] == pytest.approx(fl[0], rel=1e-14) and fl[0] > 0.05   # the rising (west) face
    # smooth data: the difference is second order in the spacing
    diffs = []
    for n in (16, 32, 64):
        p = wl.cavity(n=n, nv=4)
        lin, pos = Oracle(p, mode=1), Oracle(p, mode=1, positive_faces=1)
        _, xc, _, _ = lin.geometry()
        q = np.exp(-2.0 * xc[:, 0]) * (1.2 + 0.3 * np.sin(3 * xc[:, 1]))
        c = (n // 2) + n * (n // 2)
        diffs.append(np.abs(pos.cell_faces(c, q) - lin.cell_faces(c, q)).max())
    assert diffs[0] > 0 and 3.6 < diffs[0] / diffs[1] < 4.4 and 3.6 < diffs[1] / diffs[2] < 4.4

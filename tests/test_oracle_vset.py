"""Pins of the unstructured velocity sets (the paper's unstructured, locally refined
velocity-space discretisation) in the oracle and the input generator.

- A point set that lists a tensor grid's velocities, in shuffled order, is the same quadrature:
  the oracle's GSIS step gives the tensor grid's results (rounding order only).
- The hybrid set integrates a cold wall's Maxwellian that its base grid cannot, with a small
  fraction of the velocities of a uniform grid of its finest spacing.
- Collisionless flow between a far-field reservoir and a hot wall has its exact discrete
  solution on the point set too (molecules leaving the reservoir carry its Maxwellian, those
  leaving the wall the wall Maxwellian with the density that cancels the wall's mass flux).
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2310_18916_gb300 import workloads as wl


def _tensor_points(p):
    X, Y, Z = np.meshgrid(p.vx, p.vy, p.vz, indexing="ij")
    Wt = p.wx[:, None, None] * p.wy[None, :, None] * p.wz[None, None, :]
    flat = lambda a: a.transpose(2, 1, 0).ravel()   # v = ix + nx (iy + ny iz)
    return np.stack([flat(X), flat(Y), flat(Z), flat(Wt)], axis=1)


@pytest.mark.parametrize("mode", [0, 1])
def test_point_set_of_a_tensor_grid_reproduces_the_grid(mode):
    p = wl.cavity(n=6, nv=8, Kn=0.2, lid=0.3)
    pts = _tensor_points(p)
    perm = np.random.default_rng(5).permutation(len(pts))
    q = wl.with_velocity_set(wl.cavity(n=6, nv=8, Kn=0.2, lid=0.3), pts[perm])
    a = Oracle(p, mode=mode, macro_steps=40, nthreads=1)
    b = Oracle(q, mode=mode, macro_steps=40, nthreads=1)
    for _ in range(2):
        a.step()
        b.step()
    np.testing.assert_allclose(b.W(), a.W(), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(b.half_moments(), a.half_moments(), rtol=1e-10, atol=1e-13)
    fa, fb = a.get_f()[0], b.get_f()[0]
    np.testing.assert_allclose(fb, fa[:, perm], rtol=1e-11, atol=1e-14 * np.abs(fa).max())


def _maxwellian_moments(P, rho, u, T):
    c = P[:, :3] - u
    M = rho * (np.pi * T) ** -1.5 * np.exp(-(c * c).sum(1) / T)
    w = P[:, 3]
    m0 = w @ M
    mom = (w * M) @ P[:, :3]
    e = (w * M) @ (0.5 * (c * c).sum(1))
    return abs(m0 / rho - 1), np.abs(mom / rho - u).max(), abs(e / (0.75 * rho * T) - 1)


def test_hybrid_set_resolves_a_cold_wall_that_the_base_grid_cannot():
    """Ma 4 free stream at T = 1 and a wall at T_w = 0.3 (the hypersonic cold-wall setting of
    Section 5.2): the truncation sphere is sized by the stagnation temperature, so its base grid
    (spacing 1.1) cannot integrate the wall Maxwellian (thermal speed 0.39): its moments are off
    by tens of percent.  The refined cubes bring both Maxwellians' mass, momentum and energy to
    1e-6 with fewer than 1/5 of the velocities of a uniform grid of the finest spacing."""
    U = np.array([4.0 * np.sqrt(5.0 / 6.0), 0.0, 0.0])
    base = wl.hybrid_velocity_set(U, T_inf=1.0, T_w=0.3, n_base=16, refine=1)
    assert max(_maxwellian_moments(base, 1.0, np.zeros(3), 0.3)) > 0.1
    P = wl.hybrid_velocity_set(U, T_inf=1.0, T_w=0.3, n_base=16)
    assert max(_maxwellian_moments(P, 1.0, U, 1.0)) < 1e-6
    assert max(_maxwellian_moments(P, 1.0, np.zeros(3), 0.3)) < 1e-6
    fine = np.cbrt(P[:, 3].min())
    box = (P[:, :3].max(0) - P[:, :3].min(0)).max() + fine
    assert (box / fine) ** 3 > 5 * len(P)
    assert np.all(P[:, 3] > 0)
    # total volume of the cells: the truncation sphere's (radius 5 sqrt(T_s / 2) with the
    # stagnation temperature T_s = 1 + (gamma - 1) Ma^2 / 2), to its staircase resolution
    Rv = 5.0 * np.sqrt(0.5 * (1.0 + (2.0 / 3.0) / 2.0 * 16.0))
    assert abs(P[:, 3].sum() / (4.0 / 3.0 * np.pi * Rv ** 3) - 1) < 0.1


@pytest.mark.parametrize("U", [(0.0, 0.3, 0.0), (-0.3, 0.0, 0.0)])
def test_collisionless_reservoir_and_hot_wall_on_a_point_set(U):
    p = wl.reservoir_wall(n_cells=6, nv=4, U=U, T_inf=1.0, T_w=2.0, Kn=1e9)
    P = wl.hybrid_velocity_set(np.array(U), T_inf=1.0, T_w=2.0, n_base=14)
    p = wl.with_velocity_set(p, P)
    W0 = np.tile([0.5, 0.0, 0.0, 0.0, 1.5, 1.5], (p.ncells, 1))
    o = Oracle(p, W0=W0, mode=1)
    o.step(4)
    f, _ = o.get_f()
    xi = P[:, :3]
    M = lambda rho, u, T: rho * (np.pi * T) ** -1.5 * np.exp(-((xi - np.asarray(u)) ** 2).sum(1) / T)
    Minf, Mw = M(1.0, U, 1.0), M(1.0, (0.0, 0.0, 0.0), 2.0)
    w, vx = P[:, 3], xi[:, 0]
    up, dn = vx > 0, vx < 0
    rho_w = (w[up] * vx[up] * Minf[up]).sum() / (w[dn] * -vx[dn] * Mw[dn]).sum()
    exact = np.where(up, Minf, rho_w * Mw)
    assert np.abs(f - exact[None, :]).max() < 1e-6 * np.abs(exact).max()


def test_clustered_velocity_grid_integrates_the_free_stream_and_the_wall():
    """The stretched velocity grid of the sphere configuration (48 nodes on [-12, 12] per axis,
    clustered about the Ma-4 free-stream component): nodes increase, weights sum to the interval
    (to the midpoint rule's own error),
    spacing is finest at the free-stream velocity, and the Maxwellians of the free stream and of
    the wall at rest integrate to 1e-12 (mass, mean, variance), the 6.3 T0 post-shock gas to the
    truncation of the interval (1e-7)."""
    U = 4.0 * np.sqrt(5.0 / 6.0)
    x, w = wl.clustered_grid(48, -12.0, 12.0, U)
    assert np.all(np.diff(x) > 0) and x[0] > -12.0 and x[-1] < 12.0
    assert abs(w.sum() - 24.0) < 1e-2   # the midpoint rule for the interval's own length
    k = np.argmin(np.abs(x - U))
    assert np.diff(x)[max(k - 1, 0)] < 0.5 * np.diff(x).max()
    for T, u, tol in ((1.0, U, 1e-12), (1.0, 0.0, 1e-12), (6.3, U / 3.37, 1e-7)):
        c = x - u
        M = np.exp(-c * c / T) / np.sqrt(np.pi * T)
        assert abs(w @ M - 1) < tol and abs(w @ (M * x) - u) < tol and abs(w @ (M * c * c) - T / 2) < tol

"""Pins of the oracle on unstructured meshes (Section 5's tetrahedral, prismatic and hexahedral
cells): geometry against the closed forms, the least-squares gradient on linear fields, a
resting equilibrium that stays, the unstructured form of a structured block reaching the
structured solve's fixed point, a hybrid triangle/quadrilateral cavity converging towards the
structured cavity's solution under refinement, and GSIS on prisms and tetrahedra reaching the
kinetic iteration's fixed point."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2310_18916_gb300 import workloads as wl


def test_geometry_of_tetrahedral_and_hybrid_meshes():
    t = wl.tet_box(n=3, nv=4)
    vol, xc, S, xf = Oracle(t, mode=1, nthreads=1).geometry()
    assert len(vol) == 6 * 27
    np.testing.assert_allclose(vol, 1.0 / (6 * 27), rtol=1e-12)   # the Kuhn tetrahedra of a cube are congruent
    assert np.abs(S.sum(axis=1)).max() < 1e-15
    assert ((np.linalg.norm(S, axis=2) > 0).sum(axis=1) == 4).all()   # four faces each
    h = wl.unstructured_cavity(n=8, nv=4, hybrid=0.5)
    vol, xc, S, xf = Oracle(h, mode=1, nthreads=1).geometry()
    assert len(vol) == 8 * 4 * 2 + 8 * 4
    assert abs(vol.sum() - 1.0 / 8) < 1e-15
    assert np.abs(S.sum(axis=1)).max() < 1e-15


def test_least_squares_gradient_is_exact_for_linear_fields():
    """Cells whose face neighbours span the space: the fit of a linear field is exact."""
    for p, dims in ((wl.tet_box(n=3, nv=4), 3), (wl.unstructured_cavity(n=6, nv=4, hybrid=0.5), 2)):
        o = Oracle(p, mode=1, nthreads=1)
        vol, xc, S, xf = o.geometry()
        gvec = np.array([0.3, -1.7, 0.9])[:dims]
        q = xc[:, :dims] @ gvec + 2.5
        checked = 0
        for c in range(p.ncells):
            nb = [xc[j] - xc[c] for j in range(p.ncells)
                  if any(np.allclose(xf[c, s], xf[j, t]) for s in range(6) for t in range(6)
                         if np.linalg.norm(S[c, s]) > 0 and np.linalg.norm(S[j, t]) > 0) and j != c]
            if np.linalg.matrix_rank(np.array(nb)[:, :dims]) < dims:
                continue
            g = o.cell_gradient(c, q)
            np.testing.assert_allclose(g[:dims], gvec, rtol=0, atol=1e-11)
            checked += 1
        assert checked > p.ncells // 2


def test_resting_equilibrium_stays_on_a_tetrahedral_mesh():
    """Gas at rest in equilibrium with walls at its temperature: transport cancels on every
    closed cell and the walls re-emit what reaches them, so one step changes f only by the
    quadrature error of the collision term (3e-11 on 24^3 velocities over [-7, 7]; the structured
    box drifts the same 1.7e-6 as this mesh on 16^3 over [-6, 6])."""
    p = wl.tet_box(n=2, nv=24, vmax=7.0, wall_speed=0.0)
    o = Oracle(p, mode=1, nthreads=4)
    f0 = o.get_f()[0]
    o.step()
    assert np.abs(o.get_f()[0] - f0).max() < 1e-9 * np.abs(f0).max()


@pytest.mark.parametrize("make", ["cavity", "cylinder"])
def test_unstructured_form_reaches_the_structured_fixed_point(make):
    """The same cells given as an unstructured mesh: another sweep order (greedy colours in
    place of hyperplanes and red/black), the same discrete equations, so GSIS converges to the
    structured solve's state.  Two fixed points do not depend on the sweeps: the plain kinetic
    iteration's in an open domain (the cylinder, two passes on both forms), and GSIS with the
    implicit system solved (the cavity: the rectilinear one-pass sweep against eight greedy
    passes).  A GSIS step with an inexact implicit solve, or the closed-domain mass scale with
    the lagged wall re-emission, moves the fixed point with the number of passes (1e-6 .. 1e-5
    for two passes on these cases)."""
    if make == "cavity":
        p, sw, mode = wl.cavity(n=8, nv=12, Kn=0.3, lid=0.3), (1, 8), 0
    else:
        p, sw, mode = wl.cylinder(n_r=5, n_theta=10, nv=12, R=0.5, R_out=3.0, Ma=0.5, Kn=0.3), (2, 2), 1
    q = wl.as_unstructured(p)
    out = []
    for prob, sweeps in ((p, sw[0]), (q, sw[1])):
        o = Oracle(prob, mode=mode, n_sweeps=sweeps, macro_tol=1e-13, nthreads=4)
        o.presteps(5)
        for _ in range(400):
            if o.step() < 1e-12:
                break
        assert o.eps < 1e-12
        out.append(o.W())
    live = [0, 1, 2, 4, 5] if make == "cavity" else [0, 1, 2, 4, 5]   # u_z vanishes in these 2D flows
    scale = np.abs(out[0][:, live]).max(axis=0)
    assert (np.abs(out[1][:, live] - out[0][:, live]) / scale).max() < 1e-8


def test_hybrid_cavity_approaches_the_structured_cavity_under_refinement():
    """Different meshes of the same cavity (half triangles, half squares against squares), the
    kinetic iteration to its steady state: the shear force on the lid agrees within the
    discretisation error, which shrinks from 8^2 to 16^2."""
    diffs = []
    for n in (8, 16):
        forces = []
        for p in (wl.cavity(n=n, nv=12, Kn=0.3, lid=0.3), wl.unstructured_cavity(n=n, nv=12, Kn=0.3, lid=0.3)):
            o = Oracle(p, mode=1, n_sweeps=4 if p.ucells is not None else 1, nthreads=4)
            for _ in range(300):
                if o.step() < 1e-8:
                    break
            assert o.eps < 1e-8
            cell, side, rw, fl = o.wall()
            lid = side == 3 if p.ucells is None else np.array([p.upatch[c, s] == 3 for c, s in zip(cell, side)])
            forces.append(fl[lid, 1].sum())
        diffs.append(abs(forces[1] / forces[0] - 1))
    assert diffs[0] < 0.1 and diffs[1] < diffs[0]


@pytest.mark.parametrize("make", ["hybrid", "tetrahedra"])
def test_gsis_reaches_the_kinetic_fixed_point_on_simplices(make):
    """GSIS on meshes with prisms and tetrahedra (the synthetic solve's gradients over the
    node-sharing stencils): its converged state is the plain kinetic iteration's, reached in
    fewer than half the steps.  Both closed domains take eight passes, so that the mass scale's
    lagged wall re-emission leaves the fixed points alone, and 16 velocities per axis, on which the
    discrete reference distribution conserves to 1e-9 (with 8 to 12 the two states differ by
    that quadrature error, 1e-4 and more)."""
    if make == "hybrid":
        p = wl.unstructured_cavity(n=6, nv=16, hybrid=0.5, Kn=0.2, lid=0.3)
    else:
        p = wl.tet_box(n=2, nv=16, Kn=0.2, wall_speed=0.3)
    out, steps = [], []
    for mode in (0, 1):
        o = Oracle(p, mode=mode, n_sweeps=8, nthreads=4)
        for i in range(300):
            if o.step() < 1e-10:
                break
        assert o.eps < 1e-10
        out.append(o.W())
        steps.append(i + 1)
    scale = np.maximum(np.abs(out[1]).max(axis=0), 1e-3)
    assert (np.abs(out[0] - out[1]) / scale).max() < 5e-8
    assert 2 * steps[0] < steps[1]


def _interior_faces(o, p, k=6):
    """Up to k (cell, side) pairs of faces between two cells (no boundary patch, an area)."""
    S = o.geometry()[2]
    out = []
    for c in range(p.ucells.shape[0]):
        for s in range(6):
            if p.upatch[c, s] < 0 and np.abs(S[c, s]).max() > 0 and len(out) < k:
                out.append((c, s))
    return out


def _state(xc, u, T):
    """Conservative Shakhov state (rho = 1) of a velocity field u [cell][3] and temperature T."""
    W = np.zeros((xc.shape[0], 6))
    W[:, 0] = 1.0
    W[:, 1:4] = u
    W[:, 4] = 0.5 * (u ** 2).sum(axis=1) + 0.75 * T
    return W


def test_viscous_face_gradient_jump_term():
    """The synthetic solve's viscous face gradients on tetrahedra (reading of the face gradient
    for meshes with simplices): grad_f = mean + alpha (phi_j - phi_i - mean . d) d / |d|^2.
    - A linear field has no jump: the face stresses and heat fluxes do not depend on alpha.
    - With u = (x^2, 0, 0) at uniform T, sigma_xx, sigma_xy, sigma_xz give -mu grad_f u_x; with
      alpha = 1 its change along every centre line d equals u_x,j - u_x,i, so
      (3/4 sigma_xx, sigma_xy, sigma_xz) . d / (u_x,j - u_x,i) is the same -mu on every face
      (a reversed d or a missing 1/|d| would make it vary with the face).
    - The stress is affine in alpha, and the default weight is 1/4 on simplices."""
    p = wl.tet_box(n=3, nv=4, Kn=0.2)
    probe = Oracle(p, mode=0, nthreads=1)
    vol, xc, S, xf = probe.geometry()
    faces = _interior_faces(probe, p, k=12)
    nbr = {}
    for c, s in faces:
        # the neighbour across (c, s): the other cell with a face centred there
        hit = np.argwhere(np.abs(xf - xf[c, s]).max(axis=2) < 1e-12)
        nbr[(c, s)] = int(next(o for o, t in hit if o != c))
    A = np.array([[0.02, -0.05, 0.01], [0.03, 0.04, -0.02], [-0.01, 0.02, 0.03]])
    lin = _state(xc, xc @ A.T + 0.1, 1.0 + 0.05 * xc @ np.array([1.0, -0.5, 0.3]))
    quad = _state(xc, np.stack([0.2 * xc[:, 0] ** 2, 0 * xc[:, 0], 0 * xc[:, 0]], axis=1), np.ones(len(xc)))
    o = {a: Oracle(p, mode=0, nthreads=1, visc_jump=a) for a in (0.0, 0.25, 1.0)}
    dflt = Oracle(p, mode=0, nthreads=1)
    mus = []
    for c, s in faces:
        base = o[0.0].face_nsf(lin, c, s)
        for a in (0.25, 1.0):
            np.testing.assert_allclose(o[a].face_nsf(lin, c, s), base, rtol=1e-10, atol=1e-13)
        q0, q1, qq = (o[a].face_nsf(quad, c, s) for a in (0.0, 1.0, 0.25))
        np.testing.assert_allclose(qq, 0.75 * q0 + 0.25 * q1, rtol=1e-12, atol=1e-15)
        np.testing.assert_array_equal(dflt.face_nsf(quad, c, s), qq)
        j = nbr[(c, s)]
        d = xc[j] - xc[c]
        dphi = quad[j, 1] - quad[c, 1]
        if abs(dphi) > 1e-6:
            v = np.array([0.75 * q1[0], q1[3], q1[4]])
            mus.append(v @ d / dphi)
    assert len(mus) >= 6
    np.testing.assert_allclose(mus, mus[0], rtol=1e-10)
    assert mus[0] < 0


def test_jump_term_keeps_the_synthetic_solve_stable_on_triangles():
    """A 16 x 16 cavity of prisms and hexahedra at Kn 0.2: with the mean face gradients alone the
    synthetic solve's inner iteration diverges in the first outer step; with the default weight
    GSIS converges in under 40 steps."""
    p = wl.unstructured_cavity(n=16, nv=12, Kn=0.2, lid=0.16, hybrid=0.5)
    o = Oracle(p, mode=0, n_sweeps=4, visc_jump=0.0, nthreads=4)
    with pytest.raises(RuntimeError):
        o.step()
    o = Oracle(p, mode=0, n_sweeps=4, nthreads=4)
    for i in range(40):
        if o.step() < 1e-8:
            break
    assert o.eps < 1e-8


def test_upwind_ordered_sweeps_let_gsis_converge_on_finer_hybrid_meshes():
    """Each octant sweeps the unstructured cells in its own upwind order (ranked by the cell's
    projection on the octant's diagonal, colours one above the earlier neighbours'): on a 24 x 24
    hybrid cavity two passes carry the kinetic step close enough to steady that GSIS converges
    geometrically (the same order for every octant, a greedy colouring, stalled at eps ~ 3e-2 on
    32 x 32 and diverged on 64 x 64)."""
    p = wl.unstructured_cavity(n=24, nv=10, Kn=0.1, lid=0.16, hybrid=0.5)
    o = Oracle(p, mode=0, n_sweeps=2, nthreads=4)
    for i in range(30):
        if o.step() < 1e-8:
            break
    assert o.eps < 1e-8 and i < 25

"""Input validation at the boundary, without a GPU: gsis_footprint_bytes runs the same checks and
set-up as gsis_create, so every rejected input returns its documented error code and nothing is
allocated or launched."""
import dataclasses

import numpy as np
import pytest

from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl

GSIS_E_INVALID = -1


def code(problem, **kw):
    try:
        gsis.footprint_bytes(problem, **kw)
    except gsis.GsisError as e:
        return e.code
    return gsis.GSIS_OK


def test_valid_problems_pass():
    for p in (wl.couette(n_cells=12, nv=8), wl.cavity(n=8, nv=8), wl.box3d(ni=4, nj=3, nk=3, nv=8),
              wl.as_rykov(wl.cavity(n=6, nv=8))):
        assert code(p) == gsis.GSIS_OK, p.name


def test_curved_mesh_takes_the_general_path():
    p = wl.cavity(n=8, nv=8)
    nodes = p.nodes.copy()
    nodes[..., 0] += 0.01 * nodes[..., 1]  # x depends on J: not rectilinear
    q = dataclasses.replace(p, nodes=nodes)
    assert code(q) == gsis.GSIS_OK and code(q, mode=gsis.MODE_DVM) == gsis.GSIS_OK


def test_non_increasing_nodes_are_rejected():
    p = wl.cavity(n=8, nv=8)
    nodes = p.nodes.copy()
    nodes[..., 3, 0] = nodes[..., 2, 0]  # a zero-width cell along x
    assert code(dataclasses.replace(p, nodes=nodes)) == GSIS_E_INVALID


def test_boundary_conditions_must_match_the_axis():
    p = wl.cavity(n=8, nv=8)
    bc = list(p.bc)
    bc[0] = wl.PERIODIC  # a periodic axis is periodic on both sides
    assert code(dataclasses.replace(p, bc=bc)) == GSIS_E_INVALID
    bc[1] = wl.PERIODIC  # a wrapped axis takes the general path
    assert code(dataclasses.replace(p, bc=bc)) == gsis.GSIS_OK
    assert code(dataclasses.replace(p, bc=bc), shard=(0, 2)) == gsis.GSIS_OK
    bc = list(p.bc)
    bc[4] = wl.WALL  # an axis with one cell must be PERIODIC on both sides
    assert code(dataclasses.replace(p, bc=bc)) == GSIS_E_INVALID
    bc = list(p.bc)
    bc[1] = 7  # not a boundary condition
    assert code(dataclasses.replace(p, bc=bc), mode=gsis.MODE_DVM) == GSIS_E_INVALID


def test_general_meshes_are_accepted():
    """O-grids (far field, pole and wrapped sides) are accepted in both modes, with several colour
    passes, and velocity-sharded."""
    for p in (wl.cylinder(n_r=6, n_theta=12, nv=8), wl.sphere(n_r=4, n_pol=4, n_az=6, nv=8),
              wl.reservoir_wall(n_cells=6, nv=8)):
        assert code(p, mode=gsis.MODE_DVM, n_sweeps=3) == gsis.GSIS_OK, p.name
        assert code(p) == gsis.GSIS_OK, p.name
        assert code(p, shard=(0, 2)) == gsis.GSIS_OK, p.name
        # the synthetic solve's work arrays count in GSIS mode only
        assert gsis.footprint_bytes(p) > gsis.footprint_bytes(p, mode=gsis.MODE_DVM), p.name
        assert code(p, mode=gsis.MODE_DVM, n_sweeps=0) == GSIS_E_INVALID, p.name
    p = wl.cylinder(n_r=6, n_theta=12, nv=8)
    nodes = p.nodes.copy()
    nodes[:, :, 0, :] = nodes[:, :, 1, :]  # the first ring of cells collapses to zero volume
    assert code(dataclasses.replace(p, nodes=nodes), mode=gsis.MODE_DVM) == GSIS_E_INVALID


def test_inactive_axis_before_an_active_one_is_unsupported():
    dx = 1.0 / 8
    nodes = wl.box_nodes(np.linspace(0, 1, 9), [0.0, dx], np.linspace(0, 1, 9))
    p = wl.cavity(n=8, nv=8)
    q = dataclasses.replace(p, nj=1, nk=8, nodes=nodes,
                            bc=[wl.WALL, wl.WALL, wl.PERIODIC, wl.PERIODIC, wl.WALL, wl.WALL],
                            W0=np.tile(p.W0[:1], (64, 1)))
    assert code(q) == gsis.GSIS_E_UNSUPPORTED


def test_bad_velocity_grid_and_gas_are_rejected():
    p = wl.cavity(n=6, nv=8)
    assert code(dataclasses.replace(p, vx=p.vx[:0], wx=p.wx[:0])) == GSIS_E_INVALID
    r = wl.as_rykov(p)
    assert code(dataclasses.replace(r, d_r=0.0)) == GSIS_E_INVALID
    assert code(dataclasses.replace(r, Z_r=-1.0)) == GSIS_E_INVALID


def test_bad_shard_options_are_rejected():
    p = wl.cavity(n=6, nv=8)
    assert code(p, shard=(2, 2)) == GSIS_E_INVALID   # index outside [0, count)
    assert code(p, shard=(0, 10 ** 6)) == GSIS_E_INVALID  # more shards than velocity blocks


def test_kinetic_ring_placement():
    """The kinetic sweep's colour ring moves to a device scratch (counted in the footprint) only
    when the largest colour does not fit in shared memory, or when asked to."""
    small = wl.box3d(ni=8, nj=8, nk=8, nv=8)
    f_auto, f_global = gsis.footprint_bytes(small), gsis.footprint_bytes(small, kinetic_ring=1)
    assert f_global > f_auto
    for p, prec in ((wl.box3d(ni=20, nj=20, nk=20, nv=8), "f32"), (wl.box3d(ni=16, nj=16, nk=16, nv=8), "f64")):
        assert gsis.footprint_bytes(p, prec) == gsis.footprint_bytes(p, prec, kinetic_ring=1), p.name
    assert code(small, kinetic_ring=2) == GSIS_E_INVALID


def test_pseudo_time_step_only_in_the_kinetic_iteration():
    p = wl.cavity(n=6, nv=8)
    assert code(p, mode=gsis.MODE_DVM, kin_inv_dt=10.0) == gsis.GSIS_OK
    assert code(p, kin_inv_dt=10.0) == gsis.GSIS_E_UNSUPPORTED
    assert code(p, mode=gsis.MODE_DVM, kin_inv_dt=-1.0) == GSIS_E_INVALID


def test_euler_presteps_on_general_meshes_only():
    assert code(wl.cylinder(n_r=6, n_theta=12, nv=8), euler_presteps=100) == gsis.GSIS_OK
    assert code(wl.cavity(n=6, nv=8), euler_presteps=100) == gsis.GSIS_E_UNSUPPORTED
    assert code(wl.cylinder(n_r=6, n_theta=12, nv=8), euler_presteps=-1) == GSIS_E_INVALID


def test_odd_wrapped_axis_only_in_the_kinetic_iteration():
    """The synthetic solve's red/black colouring needs an even cell count on a wrapped axis
    (across the wrap of an odd one two neighbours would share a colour); the kinetic colours do
    not."""
    p = wl.cylinder(n_r=6, n_theta=11, nv=8)
    assert code(p) == gsis.GSIS_E_UNSUPPORTED
    assert code(p, mode=gsis.MODE_DVM) == gsis.GSIS_OK
    assert code(p, mode=gsis.MODE_DVM, euler_presteps=10) == gsis.GSIS_E_UNSUPPORTED


def _create_rc(p, Ma):
    """gsis_create through the C ABI with a given Ma; only for inputs refused before any CUDA call."""
    import ctypes as C

    L = gsis.load()
    keep = []
    m, vg, g = gsis.build_structs(p, keep)
    o = gsis.Options()
    L.gsis_default_options(C.byref(o))
    h = C.c_void_p(0)
    rc = L.gsis_create(C.byref(m), C.byref(vg), C.byref(g), float(p.Kn), float(Ma), C.byref(o), C.byref(h))
    assert not h.value
    return rc, L.gsis_last_error(None).decode()


def test_mach_number_must_match_the_free_stream_or_wall_speed():
    """gsis_create takes Ma of the free stream or of the lid (Section 5 states cases by Ma) and
    refuses a value the mesh's speeds contradict, before allocating anything."""
    cav = wl.cavity(n=8, nv=8, lid=0.16)
    assert cav.Ma == pytest.approx(0.16 / np.sqrt(5.0 / 6.0), rel=1e-14)
    for wrong in (0.0, 0.2, -0.16, float("nan")):
        rc, msg = _create_rc(cav, wrong)
        assert rc == GSIS_E_INVALID and "Ma" in msg, (wrong, rc, msg)
    cyl = wl.cylinder(n_r=4, n_theta=8, nv=8, Ma=2.0)
    assert cyl.Ma == pytest.approx(2.0, rel=1e-14)
    assert _create_rc(cyl, 2.1)[0] == GSIS_E_INVALID
    assert _create_rc(cyl, 1.0)[0] == GSIS_E_INVALID
    # the same speeds in the diatomic gas: gamma = 7/5 gives a higher Mach number
    ry = wl.as_rykov(wl.cylinder(n_r=4, n_theta=8, nv=8, Ma=2.0))
    assert ry.Ma == pytest.approx(2.0 * np.sqrt((5.0 / 3.0) / (7.0 / 5.0)), rel=1e-14)
    rc, msg = _create_rc(ry, 2.0)
    assert rc == GSIS_E_INVALID and "disagrees" in msg


def test_unstructured_velocity_sets_are_validated():
    p = wl.with_velocity_set(wl.cavity(n=8, nv=4), wl.hybrid_velocity_set((0.2, 0.0, 0.0), n_base=8, refine=2))
    assert code(p) == gsis.GSIS_OK
    for bad in (np.nan, -1.0, 0.0):
        q = wl.with_velocity_set(wl.cavity(n=8, nv=4), p.vpoints.copy())
        q.vpoints[3, 3] = bad
        assert code(q) == GSIS_E_INVALID, bad
    q = wl.with_velocity_set(wl.cavity(n=8, nv=4), p.vpoints.copy())
    q.vpoints[5, 1] = np.inf
    assert code(q) == GSIS_E_INVALID
    # footprints grow with the padded point count, not with the ignored tensor axes
    big = wl.with_velocity_set(wl.cavity(n=8, nv=4), np.concatenate([p.vpoints, p.vpoints + [0.01, 0, 0, 0]]))
    assert gsis.footprint_bytes(big) > gsis.footprint_bytes(p)


def test_unstructured_meshes_are_validated():
    """Unstructured cells through gsis_footprint_bytes (the same checks and set-up as
    gsis_create): shapes and shared sides accepted; a side neither shared nor on a patch, a
    shared side carrying a patch, a node id out of range and a PERIODIC patch not normal to z
    are refused; GSIS runs on every shape."""
    GSIS_E_UNSUPPORTED = -7
    good = (wl.tet_box(n=2, nv=8), wl.unstructured_cavity(n=4, nv=8), wl.as_unstructured(wl.cavity(n=6, nv=8)),
            wl.as_unstructured(wl.cylinder(n_r=4, n_theta=8, nv=8)))
    for p in good:
        assert code(p, mode=gsis.MODE_DVM) == gsis.GSIS_OK, p.name
    for p in good:
        assert code(p) == gsis.GSIS_OK, p.name
    p = wl.tet_box(n=2, nv=8)
    q = dataclasses.replace(p, upatch=p.upatch.copy())
    c, s = np.argwhere(q.upatch >= 0)[0]
    q.upatch[c, s] = -1   # a boundary side with no patch
    assert code(q, mode=gsis.MODE_DVM) == GSIS_E_INVALID
    q = dataclasses.replace(p, upatch=p.upatch.copy())
    shared = [(c, s) for c in range(q.ncells) for s in (0, 1, 2, 4) if p.upatch[c, s] < 0]
    q.upatch[shared[0]] = 1   # a shared side that also names a patch
    assert code(q, mode=gsis.MODE_DVM) == GSIS_E_INVALID
    q = dataclasses.replace(p, ucells=p.ucells.copy())
    q.ucells[3, 2] = len(p.unodes)
    assert code(q, mode=gsis.MODE_DVM) == GSIS_E_INVALID
    c2 = wl.unstructured_cavity(n=4, nv=8)
    q = dataclasses.replace(c2, bc=[wl.PERIODIC, wl.PERIODIC, wl.WALL, wl.WALL, wl.WALL, wl.WALL])
    assert code(q, mode=gsis.MODE_DVM) == GSIS_E_UNSUPPORTED


def test_positive_faces_on_general_meshes_only_and_wall_flux_values():
    assert code(wl.cavity(n=6, nv=8), positive_faces=1) == gsis.GSIS_E_UNSUPPORTED
    assert code(wl.cylinder(n_r=4, n_theta=8, nv=8), positive_faces=1) == 0
    assert code(wl.cylinder(n_r=4, n_theta=8, nv=8), positive_faces=2) == GSIS_E_INVALID
    assert code(wl.cavity(n=6, nv=8), wall_flux=1) == 0
    assert code(wl.cavity(n=6, nv=8), wall_flux=2) == GSIS_E_INVALID


def test_relaxed_update_only_on_general_meshes_and_in_range():
    assert code(wl.cavity(n=6, nv=8), relax=0.5) == gsis.GSIS_E_UNSUPPORTED
    assert code(wl.cavity(n=6, nv=8), relax=1.0) == 0
    assert code(wl.cylinder(n_r=4, n_theta=8, nv=8), relax=0.5) == 0
    assert code(wl.cylinder(n_r=4, n_theta=8, nv=8), relax=1.5) == GSIS_E_INVALID
    assert code(wl.cylinder(n_r=4, n_theta=8, nv=8), relax=-0.1) == GSIS_E_INVALID


def test_viscous_jump_weight_values():
    assert code(wl.cavity(n=6, nv=8), visc_jump=0.25) == gsis.GSIS_E_UNSUPPORTED
    assert code(wl.cavity(n=6, nv=8), visc_jump=0.0) == 0
    assert code(wl.cavity(n=6, nv=8), visc_jump=-1.0) == 0
    assert code(wl.cylinder(n_r=4, n_theta=8, nv=8), visc_jump=0.5) == 0
    assert code(wl.cylinder(n_r=4, n_theta=8, nv=8), visc_jump=1.5) == GSIS_E_INVALID
    assert code(wl.cylinder(n_r=4, n_theta=8, nv=8), visc_jump=float("nan")) == GSIS_E_INVALID


def test_capture_graphs_values():
    assert code(wl.cavity(n=6, nv=8), capture_graphs=1) == 0
    assert code(wl.cylinder(n_r=4, n_theta=8, nv=8), capture_graphs=1) == 0
    assert code(wl.cavity(n=6, nv=8), capture_graphs=2) == GSIS_E_INVALID

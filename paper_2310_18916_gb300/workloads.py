"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only builds inputs: mesh node coordinates, boundary conditions,
discrete velocity grids (nodes and quadrature weights), gas parameters and
initial macroscopic states.  It holds none of the solver's arithmetic, and both
the CUDA library and the CPU oracle consume what it returns.

Units are those of the solver: lengths in L, velocities in v0 = sqrt(2 R T0),
density in rho0 and temperature in T0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Side conditions: WALL (diffuse, wall_u / wall_T), PERIODIC (both sides of an axis; with
# several cells the axis closes on itself, as the azimuth of an O-grid), FARFIELD (free stream
# rho = 1, u = wall_u, T_t = T_r = wall_T), AXIS (a side of zero area: the pole of a sphere).
WALL, PERIODIC, FARFIELD, AXIS = 1, 2, 3, 4
SHAKHOV, RYKOV = 0, 1
# Nitrogen relaxation data of Section 5 (d_r = 2, omega = 0.74, A = Att, Atr, Art, Arr).
N2_A = (0.786, -0.201, -0.059, 0.842)


@dataclass
class Problem:
    ni: int
    nj: int
    nk: int
    nodes: np.ndarray            # (nk+1, nj+1, ni+1, 3) float64, i fastest in memory
    bc: list                     # 6 ints: x-, x+, y-, y+, z-, z+
    wall_u: np.ndarray           # (6, 3)
    wall_T: np.ndarray           # (6,)
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    wx: np.ndarray
    wy: np.ndarray
    wz: np.ndarray
    model: int = SHAKHOV
    omega: float = 0.81
    Kn: float = 0.1
    d_r: float = 0.0
    Z_r: float = 1.0
    A: tuple = (2.0 / 3.0, 0.0, 0.0, 1.0)
    W0: np.ndarray = field(default=None)   # (ncells, 6): rho, ux, uy, uz, Tt, Tr
    name: str = ""
    vpoints: np.ndarray = field(default=None)  # (nv, 4) unstructured velocity set: xi(3), weight
    unodes: np.ndarray = field(default=None)   # unstructured mesh: (nnodes, 3) node coordinates
    ucells: np.ndarray = field(default=None)   # (ncells, 8) node ids per cell (hexahedron order)
    upatch: np.ndarray = field(default=None)   # (ncells, 6) boundary patch per side, -1 if shared

    @property
    def ncells(self) -> int:
        if self.ucells is not None:
            return len(self.ucells)
        return self.ni * self.nj * self.nk

    @property
    def nvel(self) -> int:
        if self.vpoints is not None:
            return len(self.vpoints)
        return len(self.vx) * len(self.vy) * len(self.vz)

    @property
    def Ma(self) -> float:
        """The Mach number that describes this problem at the library's boundary: the free
        stream's speed over its speed of sound where the mesh has far-field sides, else the
        fastest wall's speed over the speed of sound at that wall's temperature, with
        c^2 = gamma T / 2 (T in T0, speeds in sqrt(2 R T0)) and gamma = (5 + d_r) / (3 + d_r)."""
        d_r = self.d_r if self.model == RYKOV else 0.0
        gamma = (5.0 + d_r) / (3.0 + d_r)
        used = set(range(6)) if self.upatch is None else {int(q) for q in np.unique(self.upatch) if q >= 0}
        far = [s for s in range(6) if s in used and self.bc[s] == FARFIELD]
        sides = far if far else [s for s in range(6) if s in used and self.bc[s] == WALL]
        return max([float(np.linalg.norm(self.wall_u[s])) / np.sqrt(0.5 * gamma * self.wall_T[s]) for s in sides],
                   default=0.0)


def midpoint_grid(n: int, lo: float, hi: float):
    """Uniform midpoint nodes and equal weights on [lo, hi]."""
    d = (hi - lo) / n
    x = lo + (np.arange(n) + 0.5) * d
    return x.astype(np.float64), np.full(n, d, dtype=np.float64)


def clustered_grid(n: int, lo: float, hi: float, center: float = 0.0, beta: float = 3.0):
    """n nodes on [lo, hi] clustered about `center`: the image of the uniform midpoints
    s = (k + 1/2)/n under xi(s) = center + a sinh(beta (s - s0)), with a and s0 such that
    xi(0) = lo and xi(1) = hi; weights xi'(s_k)/n (the midpoint rule in s).  One smooth map keeps
    the spectral accuracy of the midpoint rule for Maxwellians, which a map made of two pieces
    joined at the centre (a kink in its slope) loses.  Spacing grows by cosh(beta max(s0, 1-s0))
    from the centre to the ends."""
    Lm, Lp = center - lo, hi - center
    a_, b_ = 0.0, 1.0
    for _ in range(200):   # sinh(beta s0) / sinh(beta (1 - s0)) = Lm / Lp
        m = 0.5 * (a_ + b_)
        if np.sinh(beta * m) * Lp > np.sinh(beta * (1.0 - m)) * Lm:
            b_ = m
        else:
            a_ = m
    s0 = 0.5 * (a_ + b_)
    a = (Lm / np.sinh(beta * s0)) if s0 > 0 else (Lp / np.sinh(beta * (1.0 - s0)))
    s = (np.arange(n) + 0.5) / n
    return (center + a * np.sinh(beta * (s - s0))).astype(np.float64), (a * beta * np.cosh(beta * (s - s0)) / n).astype(np.float64)


def box_nodes(xs, ys, zs) -> np.ndarray:
    """Rectilinear node coordinates from per-axis node positions."""
    zz, yy, xx = np.meshgrid(np.asarray(zs, float), np.asarray(ys, float), np.asarray(xs, float), indexing="ij")
    return np.ascontiguousarray(np.stack([xx, yy, zz], axis=-1))


def _uniform_state(nc, rho=1.0, u=(0.0, 0.0, 0.0), Tt=1.0, Tr=1.0):
    W = np.zeros((nc, 6))
    W[:, 0] = rho
    W[:, 1:4] = u
    W[:, 4] = Tt
    W[:, 5] = Tr
    return W


def couette(n_cells=100, nv=24, vmax=5.0, U=0.2, Kn=0.1, omega=0.81, Tw=(1.0, 1.0)) -> Problem:
    """Planar Couette flow: plates at x = 0 and x = 1 moving at -U and +U along y, diffuse at Tw."""
    dx = 1.0 / n_cells
    nodes = box_nodes(np.linspace(0.0, 1.0, n_cells + 1), [0.0, dx], [0.0, dx])
    v, w = midpoint_grid(nv, -vmax, vmax)
    wall_u = np.zeros((6, 3))
    wall_u[0, 1] = -U
    wall_u[1, 1] = U
    wall_T = np.ones(6)
    wall_T[0], wall_T[1] = Tw
    return Problem(n_cells, 1, 1, nodes, [WALL, WALL, PERIODIC, PERIODIC, PERIODIC, PERIODIC], wall_u, wall_T,
                   v, v.copy(), v.copy(), w, w.copy(), w.copy(), SHAKHOV, omega, Kn,
                   W0=_uniform_state(n_cells), name=f"couette{n_cells}x{nv}^3")


def cavity(n=128, nv=32, vmax=5.0, lid=0.16, Kn=0.1, omega=0.81, stretch=0.0, ny=None) -> Problem:
    """Lid-driven cavity [0,1] x [0, ny/n]: lid y = top moves at +lid along x, all walls at T = 1
    (square with n x n cells unless ny is given).

    stretch > 0 clusters cells towards the walls (tanh spacing); 0 gives a uniform grid.
    """
    ny = n if ny is None else ny
    s = np.linspace(0.0, 1.0, n + 1)
    if stretch > 0:
        s = 0.5 * (1.0 + np.tanh(stretch * (2.0 * s - 1.0)) / np.tanh(stretch))
    sy = s if ny == n else np.linspace(0.0, ny / n, ny + 1)
    dz = 1.0 / n
    nodes = box_nodes(s, sy, [0.0, dz])
    v, w = midpoint_grid(nv, -vmax, vmax)
    wall_u = np.zeros((6, 3))
    wall_u[3, 0] = lid
    return Problem(n, ny, 1, nodes, [WALL, WALL, WALL, WALL, PERIODIC, PERIODIC], wall_u, np.ones(6),
                   v, v.copy(), v.copy(), w, w.copy(), w.copy(), SHAKHOV, omega, Kn,
                   W0=_uniform_state(n * ny), name=f"cavity{n}x{ny}x{nv}^3_Kn{Kn:g}")


def serving_cavity(rng, sizes=(32, 48, 64), nvs=(16, 20, 24), kn=(1e-3, 1.0), ma=(0.1, 1.0)) -> Problem:
    """One request of the serving stream: a lid-driven cavity with the spatial size and velocity
    count drawn from the lists, Kn log-uniform in kn, lid Mach number uniform in ma (lid speed
    Ma sqrt(gamma/2) in sqrt(2RT0) units, gamma = 5/3), and a velocity box of half-width
    max(5, lid + 5 sqrt(T_stag / 2)) with T_stag = 1 + (gamma - 1) Ma^2 / 2."""
    n = int(rng.choice(sizes))
    nv = int(rng.choice(nvs))
    Kn = float(np.exp(rng.uniform(np.log(kn[0]), np.log(kn[1]))))
    Ma = float(rng.uniform(ma[0], ma[1]))
    gamma = 5.0 / 3.0
    lid = Ma * np.sqrt(gamma / 2.0)
    t_stag = 1.0 + 0.5 * (gamma - 1.0) * Ma * Ma
    vmax = max(5.0, lid + 5.0 * np.sqrt(t_stag / 2.0))
    return cavity(n=n, nv=nv, vmax=vmax, lid=lid, Kn=Kn)


def serving_cylinder(rng, sizes=(32, 48, 64), nvs=(16, 20, 24), kn=(1e-3, 1.0), ma=(0.1, 1.0)) -> Problem:
    """One cylinder request of the serving stream: the cylinder of diameter 1 in cross flow on an
    O-grid of n radial x 2n azimuthal cells (n from sizes; radial spacing geometric from 0.01 of
    the diameter, far field at 10 diameters), nv^3 velocities on the velocity box of the free
    stream, Kn log-uniform in kn, Ma uniform in ma."""
    n = int(rng.choice(sizes))
    nv = int(rng.choice(nvs))
    Kn = float(np.exp(rng.uniform(np.log(kn[0]), np.log(kn[1]))))
    Ma = float(rng.uniform(ma[0], ma[1]))
    return cylinder(n_r=n, n_theta=2 * n, nv=nv, R=0.5, R_out=10.0, first=0.01, Ma=Ma, Kn=Kn)


def serving_request(rng, sizes=(32, 48, 64), nvs=(16, 20, 24), kn=(1e-3, 1.0), cavity_ma=(0.1, 5.0),
                    cylinder_ma=(0.1, 1.0), cylinder_kn_max=0.2, continuum_kn=0.05, continuum_ma=1.75, kn_dvm=0.3):
    """One request of the mixed serving stream: a cavity or a cylinder with equal odds, and the
    solver options a server would pick for it (returns (problem, options)).

    Kn is log-uniform in kn and the Mach number uniform in its range, within the region where
    the solves converge from the impulsive start (oracle and GPU probes at these resolutions):
    - cavities below Kn continuum_kn take lid Mach numbers up to continuum_ma only (at Kn ~1e-3 a
      lid at Mach 2.5 and above makes the state non-physical in the first steps);
    - cylinders stay subsonic and below Kn cylinder_kn_max (supersonic cylinders fail at
      moderate Kn in both modes; above Kn 0.3 GSIS stalls and the plain kinetic iteration loses
      positivity on the wall-resolved grids), with two colour passes per kinetic step;
    - GSIS below Kn kn_dvm, the plain kinetic iteration above (GSIS's synthetic NSF solve
      diverges on fast rarefied flows, which the kinetic iteration converges in tens of steps)."""
    if rng.uniform() < 0.5:
        Kn = float(np.exp(rng.uniform(np.log(kn[0]), np.log(kn[1]))))
        hi = cavity_ma[1] if Kn >= continuum_kn else min(cavity_ma[1], continuum_ma)
        p = serving_cavity(rng, sizes=sizes, nvs=nvs, kn=(Kn, Kn), ma=(cavity_ma[0], hi))
        opts = {}
    else:
        p = serving_cylinder(rng, sizes=sizes, nvs=nvs, kn=(kn[0], min(kn[1], cylinder_kn_max)), ma=cylinder_ma)
        opts = {"n_sweeps": 2}
    opts["mode"] = "gsis" if p.Kn < kn_dvm else "dvm"
    return p, opts


def radial_nodes(n_r, R, R_out, first=None):
    """n_r + 1 radii from R to R_out: uniform, or geometric with first spacing `first`."""
    if first is None:
        return np.linspace(R, R_out, n_r + 1)
    lo, hi = 1.0 + 1e-12, 10.0
    for _ in range(200):  # growth ratio q with first (q^n - 1) / (q - 1) = R_out - R
        q = 0.5 * (lo + hi)
        if first * (q ** n_r - 1.0) / (q - 1.0) > R_out - R:
            hi = q
        else:
            lo = q
    r = R + first * np.concatenate([[0.0], np.cumsum(q ** np.arange(n_r))])
    r[-1] = R_out
    return r


def velocity_box(U, T_stag, vmax_min=5.0):
    """Half-width of a velocity box holding the free stream and the stagnation gas."""
    return max(vmax_min, float(U) + 5.0 * np.sqrt(T_stag / 2.0))


def cylinder(n_r=16, n_theta=24, nv=16, R=0.5, R_out=5.0, first=None, Ma=0.5, Kn=0.1, omega=0.81, T_w=1.0,
             vmax=None) -> Problem:
    """Circular cylinder of radius R in a cross flow along +x: a 2D O-grid, i radial (wall at
    r = R, far field at R_out), j azimuthal (closed, PERIODIC), k the inactive span.  Free-stream
    speed Ma sqrt(gamma / 2) (gamma = 5/3), T = 1; midpoint velocity grid of half-width vmax
    (default: the velocity box of the free stream and its stagnation temperature)."""
    gamma = 5.0 / 3.0
    U = Ma * np.sqrt(gamma / 2.0)
    r = radial_nodes(n_r, R, R_out, first)
    th = 2.0 * np.pi * np.arange(n_theta + 1) / n_theta
    c, sn = np.cos(th), np.sin(th)
    c[-1], sn[-1] = c[0], sn[0]  # the closing node is the first one
    dz = float(r[1] - r[0])
    nodes = np.zeros((2, n_theta + 1, n_r + 1, 3))
    for k, z in enumerate((0.0, dz)):
        nodes[k, :, :, 0] = c[:, None] * r[None, :]
        nodes[k, :, :, 1] = sn[:, None] * r[None, :]
        nodes[k, :, :, 2] = z
    if vmax is None:
        vmax = velocity_box(U, 1.0 + 0.5 * (gamma - 1.0) * Ma * Ma)
    v, w = midpoint_grid(nv, -vmax, vmax)
    wall_u = np.zeros((6, 3))
    wall_u[1, 0] = U
    wall_T = np.ones(6)
    wall_T[0] = T_w
    return Problem(n_r, n_theta, 1, nodes, [WALL, FARFIELD, PERIODIC, PERIODIC, PERIODIC, PERIODIC], wall_u, wall_T,
                   v, v.copy(), v.copy(), w, w.copy(), w.copy(), SHAKHOV, omega, Kn,
                   W0=_uniform_state(n_r * n_theta, u=(U, 0.0, 0.0)), name=f"cylinder{n_r}x{n_theta}x{nv}^3_Ma{Ma:g}")


def sphere(n_r=8, n_pol=6, n_az=8, nv=12, R=0.5, R_out=5.0, first=None, Ma=0.5, Kn=0.1, omega=0.81, T_w=1.0,
           vmax=None) -> Problem:
    """Sphere of radius R in a flow along +x: a spherical O-grid, i radial (wall at r = R, far
    field at R_out), j polar angle from the +x axis (both ends AXIS: faces of zero area), k
    azimuth (closed, PERIODIC).  Free stream and velocity grid as for `cylinder`."""
    gamma = 5.0 / 3.0
    U = Ma * np.sqrt(gamma / 2.0)
    r = radial_nodes(n_r, R, R_out, first)
    th = np.pi * np.arange(n_pol + 1) / n_pol
    ct, st = np.cos(th), np.sin(th)
    ct[0], st[0], ct[-1], st[-1] = 1.0, 0.0, -1.0, 0.0  # the poles are single points
    ph = 2.0 * np.pi * np.arange(n_az + 1) / n_az
    cp, sp = np.cos(ph), np.sin(ph)
    cp[-1], sp[-1] = cp[0], sp[0]
    nodes = np.zeros((n_az + 1, n_pol + 1, n_r + 1, 3))
    nodes[..., 0] = ct[None, :, None] * r[None, None, :]
    nodes[..., 1] = (st[None, :, None] * cp[:, None, None]) * r[None, None, :]
    nodes[..., 2] = (st[None, :, None] * sp[:, None, None]) * r[None, None, :]
    if vmax is None:
        vmax = velocity_box(U, 1.0 + 0.5 * (gamma - 1.0) * Ma * Ma)
    v, w = midpoint_grid(nv, -vmax, vmax)
    wall_u = np.zeros((6, 3))
    wall_u[1, 0] = U
    wall_T = np.ones(6)
    wall_T[0] = T_w
    nc = n_r * n_pol * n_az
    return Problem(n_r, n_pol, n_az, nodes, [WALL, FARFIELD, AXIS, AXIS, PERIODIC, PERIODIC], wall_u, wall_T,
                   v, v.copy(), v.copy(), w, w.copy(), w.copy(), SHAKHOV, omega, Kn,
                   W0=_uniform_state(nc, u=(U, 0.0, 0.0)), name=f"sphere{n_r}x{n_pol}x{n_az}x{nv}^3_Ma{Ma:g}")


def reservoir_wall(n_cells=10, nv=16, vmax=5.0, U=(0.0, 0.3, 0.0), T_inf=1.0, T_w=2.0, Kn=1e7) -> Problem:
    """1D slab x in [0, 1]: a far field (free stream rho = 1, U, T_inf) at x = 0 and a diffuse
    wall at rest at T_w at x = 1."""
    dx = 1.0 / n_cells
    nodes = box_nodes(np.linspace(0.0, 1.0, n_cells + 1), [0.0, dx], [0.0, dx])
    v, w = midpoint_grid(nv, -vmax, vmax)
    wall_u = np.zeros((6, 3))
    wall_u[0] = U
    wall_T = np.ones(6)
    wall_T[0], wall_T[1] = T_inf, T_w
    return Problem(n_cells, 1, 1, nodes, [FARFIELD, WALL, PERIODIC, PERIODIC, PERIODIC, PERIODIC], wall_u, wall_T,
                   v, v.copy(), v.copy(), w, w.copy(), w.copy(), SHAKHOV, 0.81, Kn,
                   W0=_uniform_state(n_cells, u=U, Tt=T_inf, Tr=T_inf), name=f"reservoir{n_cells}x{nv}^3")


def box3d(ni=6, nj=5, nk=4, nv=12, vmax=5.0, Kn=0.1, omega=0.81, wall_speed=0.2) -> Problem:
    """Small closed 3D box with one moving wall (z+ moves along x); all walls diffuse at T = 1."""
    nodes = box_nodes(np.linspace(0, 1, ni + 1), np.linspace(0, 0.8, nj + 1), np.linspace(0, 0.6, nk + 1))
    v, w = midpoint_grid(nv, -vmax, vmax)
    wall_u = np.zeros((6, 3))
    wall_u[5, 0] = wall_speed
    return Problem(ni, nj, nk, nodes, [WALL] * 6, wall_u, np.ones(6), v, v.copy(), v.copy(), w, w.copy(), w.copy(),
                   SHAKHOV, omega, Kn, W0=_uniform_state(ni * nj * nk), name=f"box{ni}x{nj}x{nk}")


def as_rykov(p: Problem, d_r=2.0, Z_r=5.0, A=N2_A, omega=0.74) -> Problem:
    """The same geometry with the diatomic Rykov-type gas of Section 2.2 (nitrogen data of Section 5)."""
    p.model, p.d_r, p.Z_r, p.A, p.omega = RYKOV, d_r, Z_r, tuple(A), omega
    p.name += "_rykov"
    return p


def perturbed_state(p: Problem, seed=0, amp=0.05) -> np.ndarray:
    """Seeded smooth perturbation of the uniform initial state (rho, u, Tt, Tr per cell)."""
    rng = np.random.default_rng(seed)
    W = p.W0.copy()
    nc = p.ncells
    W[:, 0] *= 1.0 + amp * rng.uniform(-1, 1, nc)
    W[:, 1:4] += amp * rng.uniform(-1, 1, (nc, 3))
    W[:, 4] *= 1.0 + amp * rng.uniform(-1, 1, nc)
    W[:, 5] *= 1.0 + amp * rng.uniform(-1, 1, nc)
    return W


def random_vdf(p: Problem, seed=0, amp=0.1, W=None):
    """Seeded non-equilibrium VDFs [cell][v] (v = ix + nx (iy + ny iz)): a local
    Maxwellian-shaped envelope times a random positive modulation.

    The envelope is written out here only to make positive, decaying test data; it is
    an input recipe, not the solver's equilibrium routine.
    """
    rng = np.random.default_rng(seed)
    W = p.W0 if W is None else W
    VX, VY, VZ = np.meshgrid(p.vx, p.vy, p.vz, indexing="ij")
    # flatten with ix fastest: transpose (iz, iy, ix)
    X = VX.transpose(2, 1, 0).ravel()
    Y = VY.transpose(2, 1, 0).ravel()
    Z = VZ.transpose(2, 1, 0).ravel()
    nc, nv = p.ncells, p.nvel
    f0 = np.empty((nc, nv))
    for c in range(nc):
        rho, ux, uy, uz, T = W[c, 0], W[c, 1], W[c, 2], W[c, 3], W[c, 4]
        env = rho * (np.pi * T) ** -1.5 * np.exp(-((X - ux) ** 2 + (Y - uy) ** 2 + (Z - uz) ** 2) / T)
        f0[c] = env * (1.0 + amp * rng.uniform(-1, 1, nv))
    f1 = None
    if p.model == RYKOV:
        f1 = f0 * (p.d_r * W[:, 5:6] / 4.0) * (1.0 + amp * rng.uniform(-1, 1, (nc, nv)))
    return f0, f1


def hybrid_velocity_set(U=(0.0, 0.0, 0.0), T_inf=1.0, T_w=1.0, gamma=5.0 / 3.0, n_base=16, refine=3,
                        radius_sigmas=5.0, refine_sigmas=5.0):
    """Unstructured, locally refined velocity set after the paper's unstructured velocity-space
    discretisation (Section 5.2): velocity space truncated to a sphere about the post-shock velocity
    U_s = U_inf / r, r = (gamma + 1) Ma^2 / (2 + (gamma - 1) Ma^2) (taken as 1 below Ma = 1), with
    radius radius_sigmas sqrt(R T_s), T_s = max(T_inf (1 + (gamma - 1) Ma^2 / 2), T_w, T_inf); a
    Cartesian base grid of n_base cells across that diameter, keeping the cells whose centre lies in
    the sphere; every base cell that meets a refinement cube (half-width refine_sigmas sqrt(R T)
    about U_inf with T_inf and about 0 with T_w) split into refine^3 sub-cells.  Each cell gives one
    discrete velocity (its centre) with its volume as quadrature weight: the hexahedral octree
    stands in for the paper's tetrahedral filling.  The paper refines within 3 sqrt(R T); the
    default here is 5, since a refinement boundary where the Maxwellian still holds 0.3 % of its
    mass costs the midpoint rule its spectral accuracy (~1e-3 in the moments; ~1e-8 at 5).
    Units: R T = T / 2.  Returns (nv, 4) points."""
    U = np.asarray(U, dtype=float)
    Ma = float(np.linalg.norm(U)) / np.sqrt(0.5 * gamma * T_inf)
    ratio = max(1.0, (gamma + 1.0) * Ma * Ma / (2.0 + (gamma - 1.0) * Ma * Ma)) if Ma > 0 else 1.0
    Us = U / ratio
    Ts = max(T_inf * (1.0 + 0.5 * (gamma - 1.0) * Ma * Ma), T_w, T_inf)
    Rv = radius_sigmas * np.sqrt(0.5 * Ts)
    h = 2.0 * Rv / n_base
    cubes = [(U, refine_sigmas * np.sqrt(0.5 * T_inf)), (np.zeros(3), refine_sigmas * np.sqrt(0.5 * T_w))]
    i = np.arange(n_base) + 0.5 - 0.5 * n_base
    C = np.stack(np.meshgrid(i, i, i, indexing="ij"), -1).reshape(-1, 3) * h + Us
    C = C[np.linalg.norm(C - Us, axis=1) <= Rv]
    fine = np.zeros(len(C), dtype=bool)
    for P, L in cubes:
        fine |= np.all(np.abs(C - P) <= L + 0.5 * h, axis=1)
    coarse = np.concatenate([C[~fine], np.full((int((~fine).sum()), 1), h ** 3)], axis=1)
    k = (np.arange(refine) + 0.5) / refine - 0.5
    sub = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3) * h
    F = (C[fine][:, None, :] + sub[None, :, :]).reshape(-1, 3)
    finep = np.concatenate([F, np.full((len(F), 1), (h / refine) ** 3)], axis=1)
    return np.ascontiguousarray(np.concatenate([coarse, finep]), dtype=np.float64)


def with_clustered_velocities(p: Problem, n: int, vmax: float, beta: float = 3.0) -> Problem:
    """The same problem on n^3 velocities over [-vmax, vmax]^3, clustered per axis about the
    free-stream (or, without a far field, the fastest wall's) velocity component."""
    far = [s for s in range(6) if p.bc[s] == FARFIELD]
    sides = far if far else [s for s in range(6) if p.bc[s] == WALL]
    U = max((p.wall_u[s] for s in sides), key=lambda u: float(np.linalg.norm(u)), default=np.zeros(3))
    grids = [clustered_grid(n, -vmax, vmax, float(U[a]), beta) for a in range(3)]
    (p.vx, p.wx), (p.vy, p.wy), (p.vz, p.wz) = grids
    p.name += f"_clustered{n}"
    return p


def with_velocity_set(p: Problem, points) -> Problem:
    """The same problem on an unstructured velocity set (points: (nv, 4) = xi(3), weight)."""
    p.vpoints = np.ascontiguousarray(points, dtype=np.float64)
    p.name += f"_vset{len(points)}"
    return p


# Sides of a hexahedral cell (corner t at offsets (t & 1, (t >> 1) & 1, t >> 2)), the order of
# the library's unstructured meshes: x-, x+, y-, y+, z-, z+ for an axis-aligned cell.
HEX_SIDES = ((0, 2, 6, 4), (1, 3, 7, 5), (0, 1, 5, 4), (2, 3, 7, 6), (0, 1, 3, 2), (4, 5, 7, 6))


def _patches_by_position(nodes, cells, box):
    """Boundary patch of each cell side from where its face lies on the axis-aligned box
    ((x0, x1), (y0, y1), (z0, z1)): 0/1 on x = x0/x1, 2/3 on y, 4/5 on z; -1 for inner sides.
    Sides whose corners span no area are left -1 (they carry no flux)."""
    patch = np.full((len(cells), 6), -1, dtype=np.int32)
    for c, ids in enumerate(cells):
        for sd, corners in enumerate(HEX_SIDES):
            q = np.array([ids[t] for t in corners])
            if len(set(q.tolist())) < 3:
                continue
            P = nodes[q]
            for a in range(3):
                for hi in range(2):
                    if np.all(np.abs(P[:, a] - box[a][hi]) < 1e-12):
                        patch[c, sd] = 2 * a + hi
    return patch


def as_unstructured(p: Problem) -> Problem:
    """The same block as an unstructured mesh: every cell a hexahedron of node ids, sides on the
    block's boundary in the patch of that side; the nodes of a closed (wrapped) axis merged.  A
    one-cell periodic axis becomes a one-layer PERIODIC patch and must lie along z."""
    ni, nj, nk = p.ni, p.nj, p.nk
    n = (ni, nj, nk)
    wrap = [p.bc[2 * a] == PERIODIC and n[a] >= 3 for a in range(3)]
    N = (ni + 1, nj + 1, nk + 1)
    X = p.nodes.reshape(-1, 3)
    def nid(I, J, K):
        I, J, K = [q % n[a] if wrap[a] else q for a, q in enumerate((I, J, K))]
        return I + N[0] * (J + N[1] * K)
    cells, patch = [], []
    for k in range(nk):
        for j in range(nj):
            for i in range(ni):
                cells.append([nid(i + (t & 1), j + ((t >> 1) & 1), k + (t >> 2)) for t in range(8)])
                idx = (i, j, k)
                pt = []
                for sd in range(6):
                    a, hi = sd // 2, sd & 1
                    at_edge = idx[a] == (n[a] - 1 if hi else 0)
                    pt.append(sd if at_edge and not wrap[a] else -1)
                patch.append(pt)
    q = Problem(ni, nj, nk, p.nodes, list(p.bc), p.wall_u.copy(), p.wall_T.copy(), p.vx, p.vy, p.vz, p.wx, p.wy, p.wz,
                p.model, p.omega, p.Kn, p.d_r, p.Z_r, p.A, p.W0, p.name + "_unstructured", p.vpoints)
    q.unodes = np.ascontiguousarray(X, dtype=np.float64)
    q.ucells = np.ascontiguousarray(cells, dtype=np.int32)
    q.upatch = np.ascontiguousarray(patch, dtype=np.int32)
    return q


def unstructured_cavity(n=8, nv=12, vmax=5.0, lid=0.16, Kn=0.1, omega=0.81, hybrid=0.5) -> Problem:
    """The lid-driven cavity [0, 1]^2 as a one-layer unstructured mesh: the n x n squares with
    x < hybrid split into two triangles each (alternating diagonals), the others kept whole;
    extruded one cell in z (prisms and hexahedra sharing quadrilateral faces).  Walls on the
    four sides (patches 0..3, the lid y = 1 moving along x), a PERIODIC patch on the two z faces."""
    xs = np.linspace(0.0, 1.0, n + 1)
    dz = 1.0 / n
    nid = lambda i, j, k: i + (n + 1) * (j + (n + 1) * k)
    nodes = np.array([[xs[i], xs[j], k * dz] for k in range(2) for j in range(n + 1) for i in range(n + 1)])
    cells = []
    for j in range(n):
        for i in range(n):
            a, b, c, d = nid(i, j, 0), nid(i + 1, j, 0), nid(i, j + 1, 0), nid(i + 1, j + 1, 0)
            A_, B_, C_, D_ = a + (n + 1) ** 2, b + (n + 1) ** 2, c + (n + 1) ** 2, d + (n + 1) ** 2
            if (i + 0.5) / n < hybrid:
                tris = ((a, b, d), (a, d, c)) if (i + j) % 2 == 0 else ((a, b, c), (b, d, c))
                top = {a: A_, b: B_, c: C_, d: D_}
                for t0, t1, t2 in tris:
                    cells.append([t0, t1, t2, t2, top[t0], top[t1], top[t2], top[t2]])
            else:
                cells.append([a, b, c, d, A_, B_, C_, D_])
    cells = np.array(cells, dtype=np.int32)
    patch = _patches_by_position(nodes, cells, ((0.0, 1.0), (0.0, 1.0), (0.0, dz)))
    v, w = midpoint_grid(nv, -vmax, vmax)
    wall_u = np.zeros((6, 3))
    wall_u[3, 0] = lid
    p = Problem(1, 1, 1, np.zeros((2, 2, 2, 3)), [WALL, WALL, WALL, WALL, PERIODIC, PERIODIC], wall_u, np.ones(6), v,
                v.copy(), v.copy(), w, w.copy(), w.copy(), SHAKHOV, omega, Kn, W0=_uniform_state(len(cells)),
                name=f"ucavity{n}x{nv}^3_h{hybrid:g}")
    p.unodes, p.ucells, p.upatch = np.ascontiguousarray(nodes), cells, patch
    return p


def tet_box(n=3, nv=8, vmax=5.0, Kn=0.1, omega=0.81, wall_speed=0.2) -> Problem:
    """The unit cube with diffuse walls (the z = 1 wall moving along x), its n^3 cubes each split
    into six tetrahedra along the main diagonal (the Kuhn split: conforming across cubes)."""
    import itertools

    nid = lambda i, j, k: i + (n + 1) * (j + (n + 1) * k)
    h = 1.0 / n
    nodes = np.array([[i * h, j * h, k * h] for k in range(n + 1) for j in range(n + 1) for i in range(n + 1)])
    cells = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                for perm in itertools.permutations(range(3)):
                    cur = [i, j, k]
                    path = [nid(*cur)]
                    for ax in perm:
                        cur[ax] += 1
                        path.append(nid(*cur))
                    a, b, c, d = path
                    cells.append([a, b, c, c, d, d, d, d])
    cells = np.array(cells, dtype=np.int32)
    patch = _patches_by_position(nodes, cells, ((0.0, 1.0), (0.0, 1.0), (0.0, 1.0)))
    v, w = midpoint_grid(nv, -vmax, vmax)
    wall_u = np.zeros((6, 3))
    wall_u[5, 0] = wall_speed
    p = Problem(1, 1, 1, np.zeros((2, 2, 2, 3)), [WALL] * 6, wall_u, np.ones(6), v, v.copy(), v.copy(), w, w.copy(),
                w.copy(), SHAKHOV, omega, Kn, W0=_uniform_state(len(cells)), name=f"tetbox{n}x{nv}^3")
    p.unodes, p.ucells, p.upatch = np.ascontiguousarray(nodes), cells, patch
    return p


def capsule_profile(theta, x_o=-0.2, cap_half_angle=np.pi / 3, cone_half_angle=np.radians(33.0)):
    """Distance from the origin (x_o, 0) to the capsule's surface along the meridian ray at polar
    angle theta from +x: a spherical-cap heat shield of radius 1 centred at the origin of x, facing
    -x, up to the shoulder at cap_half_angle from the -x axis, then a cone converging downstream at
    cone_half_angle to its apex on the axis."""
    c, s = np.cos(theta), np.sin(theta)
    # the cap: |(x_o + t c, t s)| = 1
    b = x_o * c
    t_cap = -b + np.sqrt(b * b - x_o * x_o + 1.0)
    xs, ys = -np.cos(cap_half_angle), np.sin(cap_half_angle)        # the shoulder
    xa = xs + ys / np.tan(cone_half_angle)                          # the apex
    # the cone: points (x, y) with y = (xa - x) tan(cone_half_angle), x in [xs, xa]
    k = np.tan(cone_half_angle)
    t_cone = (xa - x_o) * k / (s + c * k)
    x_cap = x_o + t_cap * c
    return np.where(x_cap <= xs, t_cap, t_cone)


def capsule(n_r=50, n_pol=40, n_az=50, nv=48, R_out=6.0, first=None, Ma=10.0, Kn=0.01, T_w=0.3, vmax=None,
            rykov=True) -> Problem:
    """Hypersonic capsule forebody in a flow along +x: the body of revolution of capsule_profile
    (heat-shield cap radius 1, 33 deg conical afterbody), a spherical O-grid about (-0.2, 0, 0):
    i radial from the body (diffuse wall at T_w) to a far field at R_out, j polar from +x (AXIS at
    both poles), k azimuth (closed).  The diatomic Rykov gas of Section 5 (d_r = 2, Z_r = 5,
    nitrogen A, omega 0.74) by default, free stream U = Ma sqrt(gamma T / 2) with gamma = 7/5,
    T = 1; velocities clustered about the free stream on [-vmax, vmax]^3 (default: 3.5 thermal
    speeds of the stagnation gas, and 4.5 beyond the free-stream speed)."""
    gamma = 7.0 / 5.0 if rykov else 5.0 / 3.0
    U = Ma * np.sqrt(gamma / 2.0)
    if vmax is None:
        vmax = max(U + 4.5, 3.5 * np.sqrt(1.0 + 0.5 * (gamma - 1.0) * Ma * Ma))
    th = np.pi * np.arange(n_pol + 1) / n_pol
    ct, st = np.cos(th), np.sin(th)
    ct[0], st[0], ct[-1], st[-1] = 1.0, 0.0, -1.0, 0.0
    rb = capsule_profile(th)
    ph = 2.0 * np.pi * np.arange(n_az + 1) / n_az
    cp, sp = np.cos(ph), np.sin(ph)
    cp[-1], sp[-1] = cp[0], sp[0]
    nodes = np.zeros((n_az + 1, n_pol + 1, n_r + 1, 3))
    for j in range(n_pol + 1):
        r = radial_nodes(n_r, rb[j], R_out, None if first is None else first * rb[j])
        nodes[:, j, :, 0] = -0.2 + ct[j] * r[None, :]
        nodes[:, j, :, 1] = (st[j] * cp[:, None]) * r[None, :]
        nodes[:, j, :, 2] = (st[j] * sp[:, None]) * r[None, :]
    v, w = midpoint_grid(nv, -vmax, vmax)
    wall_u = np.zeros((6, 3))
    wall_u[1, 0] = U
    wall_T = np.ones(6)
    wall_T[0] = T_w
    nc = n_r * n_pol * n_az
    p = Problem(n_r, n_pol, n_az, nodes, [WALL, FARFIELD, AXIS, AXIS, PERIODIC, PERIODIC], wall_u, wall_T,
                v, v.copy(), v.copy(), w, w.copy(), w.copy(), SHAKHOV, 0.81, Kn,
                W0=_uniform_state(nc, u=(U, 0.0, 0.0)), name=f"capsule{n_r}x{n_pol}x{n_az}_Ma{Ma:g}")
    if rykov:
        p = as_rykov(p)
    return with_clustered_velocities(p, nv, vmax)

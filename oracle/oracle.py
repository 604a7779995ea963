"""ctypes wrapper of the C oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py use it.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build_oracle

_lib = None
D = C.POINTER(C.c_double)


class OrcMesh(C.Structure):
    _fields_ = [("ni", C.c_int), ("nj", C.c_int), ("nk", C.c_int), ("nodes", D), ("bc", C.c_int * 6),
                ("wall_u", (C.c_double * 3) * 6), ("wall_T", C.c_double * 6), ("ncells", C.c_int), ("nnodes", C.c_int),
                ("unodes", D), ("cells", C.POINTER(C.c_int)), ("face_patch", C.POINTER(C.c_int))]


class OrcVgrid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("x", D * 3), ("w", D * 3), ("npoints", C.c_int), ("points", D)]


class OrcGas(C.Structure):
    _fields_ = [("model", C.c_int), ("omega", C.c_double), ("Kn", C.c_double), ("d_r", C.c_double),
                ("Z_r", C.c_double), ("A", C.c_double * 4)]


class OrcOpts(C.Structure):
    _fields_ = [("mode", C.c_int), ("schedule", C.c_int), ("n_sweeps", C.c_int), ("macro_steps", C.c_int),
                ("macro_sweeps", C.c_int), ("macro_cfl", C.c_double), ("macro_tol", C.c_double),
                ("kin_inv_dt", C.c_double), ("venkat_K", C.c_double), ("nthreads", C.c_int),
                ("wall_flux", C.c_int), ("positive_faces", C.c_int),
                ("relax", C.c_double), ("visc_jump", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        _lib = C.CDLL(path)
        L = _lib
        L.orc_create.argtypes = [C.POINTER(OrcMesh), C.POINTER(OrcVgrid), C.POINTER(OrcGas), C.POINTER(OrcOpts), D,
                                 C.POINTER(C.c_void_p)]
        L.orc_destroy.argtypes = [C.c_void_p]
        for name in ("orc_step", "orc_wall_prepass", "orc_macro_from_current", "orc_ncells", "orc_nvel",
                     "orc_nwall", "orc_macro_iters"):
            getattr(L, name).argtypes = [C.c_void_p]
        L.orc_presteps.argtypes = [C.c_void_p, C.c_int]
        L.orc_set_kin_inv_dt.argtypes = [C.c_void_p, C.c_double]
        L.orc_set_mode.argtypes = [C.c_void_p, C.c_int]
        L.orc_euler_presteps.argtypes = [C.c_void_p, C.c_int]
        L.orc_kinetic_velocities.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.orc_eps.argtypes = [C.c_void_p]
        L.orc_eps.restype = C.c_double
        L.orc_mass_scale.argtypes = [C.c_void_p]
        L.orc_mass_scale.restype = C.c_double
        L.orc_set_f.argtypes = [C.c_void_p, D, D]
        L.orc_get_f.argtypes = [C.c_void_p, D, D]
        L.orc_get_W.argtypes = [C.c_void_p, D]
        L.orc_get_half_moments.argtypes = [C.c_void_p, D]
        L.orc_get_hot.argtypes = [C.c_void_p, D]
        L.orc_get_wall.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), D, D]
        L.orc_get_geometry.argtypes = [C.c_void_p, D, D, D, D]
        L.orc_cell_gradient.argtypes = [C.c_void_p, C.c_int, D, D]
        L.orc_cell_limiter.argtypes = [C.c_void_p, C.c_int, D]
        L.orc_cell_limiter.restype = C.c_double
        L.orc_cell_faces.argtypes = [C.c_void_p, C.c_int, D, D]
        L.orc_face_nsf.argtypes = [C.c_void_p, D, C.c_int, C.c_int, D]
        L.orc_get_face_flux.argtypes = [C.c_void_p, D]
        L.orc_wall_flux.argtypes = [C.c_void_p, C.c_int, C.c_int, D, D, D, D]
        L.orc_tau.argtypes = [C.POINTER(OrcGas), C.c_double, C.c_double]
        L.orc_tau.restype = C.c_double
        L.orc_conductivity.argtypes = [C.POINTER(OrcGas), C.c_double, D, D]
        L.orc_reference.argtypes = [C.POINTER(OrcGas), D, D, D, D]
        L.orc_venkat_face.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_venkat_face.restype = C.c_double
    return _lib


def _p(a):
    return a.ctypes.data_as(D)


def gas_struct(p) -> OrcGas:
    g = OrcGas()
    g.model, g.omega, g.Kn, g.d_r, g.Z_r = p.model, p.omega, p.Kn, p.d_r, p.Z_r
    for i in range(4):
        g.A[i] = p.A[i]
    return g


DEFAULTS = dict(mode=0, schedule=0, n_sweeps=1, macro_steps=300, macro_sweeps=4, macro_cfl=100.0,
                macro_tol=1e-10, kin_inv_dt=0.0, venkat_K=1.0, nthreads=0, wall_flux=0, positive_faces=0, relax=0.0,
                visc_jump=-1.0)


class Oracle:
    """One oracle solver for a workloads.Problem."""

    def __init__(self, p, W0=None, **opts):
        L = lib()
        o = dict(DEFAULTS)
        o.update(opts)
        if o["nthreads"] <= 0:
            o["nthreads"] = os.cpu_count() or 1
        self.p = p
        self._keep = []
        nodes = np.ascontiguousarray(p.nodes, dtype=np.float64)
        self._keep.append(nodes)
        m = OrcMesh()
        m.ni, m.nj, m.nk = p.ni, p.nj, p.nk
        m.nodes = _p(nodes)
        if getattr(p, "ucells", None) is not None:
            un = np.ascontiguousarray(p.unodes, dtype=np.float64)
            uc = np.ascontiguousarray(p.ucells, dtype=np.int32)
            up = np.ascontiguousarray(p.upatch, dtype=np.int32)
            self._keep += [un, uc, up]
            m.ncells, m.nnodes = len(uc), len(un)
            m.unodes = _p(un)
            m.cells = uc.ctypes.data_as(C.POINTER(C.c_int))
            m.face_patch = up.ctypes.data_as(C.POINTER(C.c_int))
        for s in range(6):
            m.bc[s] = p.bc[s]
            m.wall_T[s] = p.wall_T[s]
            for d in range(3):
                m.wall_u[s][d] = p.wall_u[s][d]
        vg = OrcVgrid()
        for a, (x, w) in enumerate(((p.vx, p.wx), (p.vy, p.wy), (p.vz, p.wz))):
            x = np.ascontiguousarray(x, dtype=np.float64)
            w = np.ascontiguousarray(w, dtype=np.float64)
            self._keep += [x, w]
            vg.n[a] = len(x)
            vg.x[a] = _p(x)
            vg.w[a] = _p(w)
        if getattr(p, "vpoints", None) is not None:
            pts = np.ascontiguousarray(p.vpoints, dtype=np.float64)
            self._keep.append(pts)
            vg.npoints = len(pts)
            vg.points = _p(pts)
        g = gas_struct(p)
        oo = OrcOpts(**o)
        W = np.ascontiguousarray(p.W0 if W0 is None else W0, dtype=np.float64)
        h = C.c_void_p()
        rc = L.orc_create(C.byref(m), C.byref(vg), C.byref(g), C.byref(oo), _p(W), C.byref(h))
        if rc != 0:
            raise RuntimeError(f"orc_create failed: {rc}")
        self.h = h
        self.g = g
        self.nc = L.orc_ncells(h)
        self.nv = L.orc_nvel(h)
        self.nwall = L.orc_nwall(h)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def _rc(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"{what} failed: {rc}")

    def step(self, n=1):
        for _ in range(n):
            self._rc(lib().orc_step(self.h), "orc_step")
        return self.eps

    def set_kin_inv_dt(self, inv_dt):
        lib().orc_set_kin_inv_dt(self.h, float(inv_dt))

    def set_mode(self, mode):
        lib().orc_set_mode(self.h, int(mode))

    def presteps(self, n):
        self._rc(lib().orc_presteps(self.h, n), "orc_presteps")

    def euler_presteps(self, n):
        self._rc(lib().orc_euler_presteps(self.h, n), "orc_euler_presteps")

    def run(self, max_outer, tol):
        hist = []
        for _ in range(max_outer):
            hist.append(self.step())
            if hist[-1] < tol:
                break
        return hist

    def wall_prepass(self):
        self._rc(lib().orc_wall_prepass(self.h), "orc_wall_prepass")

    def kinetic_velocities(self, v0, v1):
        self._rc(lib().orc_kinetic_velocities(self.h, v0, v1), "orc_kinetic_velocities")

    def macro_from_current(self):
        self._rc(lib().orc_macro_from_current(self.h), "orc_macro_from_current")

    @property
    def eps(self):
        return lib().orc_eps(self.h)

    @property
    def mass_scale(self):
        return lib().orc_mass_scale(self.h)

    @property
    def macro_iters(self):
        return lib().orc_macro_iters(self.h)

    def set_f(self, f0, f1=None):
        f0 = np.ascontiguousarray(f0, dtype=np.float64)
        f1c = None if f1 is None else np.ascontiguousarray(f1, dtype=np.float64)
        self._rc(lib().orc_set_f(self.h, _p(f0), None if f1c is None else _p(f1c)), "orc_set_f")

    def get_f(self):
        f0 = np.empty((self.nc, self.nv))
        f1 = np.empty((self.nc, self.nv)) if self.p.model == 1 else None
        lib().orc_get_f(self.h, _p(f0), None if f1 is None else _p(f1))
        return f0, f1

    def W(self):
        out = np.empty((self.nc, 6))
        lib().orc_get_W(self.h, _p(out))
        return out

    def half_moments(self):
        out = np.empty((self.nc, 18))
        lib().orc_get_half_moments(self.h, _p(out))
        return out

    def hot(self):
        out = np.empty((self.nc, 12))
        lib().orc_get_hot(self.h, _p(out))
        return out

    def wall(self):
        n = self.nwall
        cell = np.empty(n, dtype=np.int32)
        side = np.empty(n, dtype=np.int32)
        rw = np.empty(n)
        fl = np.empty((n, 6))
        lib().orc_get_wall(self.h, cell.ctypes.data_as(C.POINTER(C.c_int)), side.ctypes.data_as(C.POINTER(C.c_int)),
                           _p(rw), _p(fl))
        return cell, side, rw, fl

    def wall_flux(self, mode, patch, pr, m18, n):
        """orc_wall_flux: the outward wall flux (rho, momentum, energy, rotational energy) of the
        state pr = (rho, u, Tt, Tr) on patch `patch` along the unit normal n; mode 0 the local
        Maxwellian, 1 the Grad-13 VDF with the stress and heat fluxes of m18."""
        out = np.zeros(6)
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (pr, m18, n)]
        lib().orc_wall_flux(self.h, int(mode), int(patch), _p(a[0]), _p(a[1]), _p(a[2]), _p(out))
        return out

    def face_flux(self):
        out = np.empty((self.nc, 6, 6))
        lib().orc_get_face_flux(self.h, _p(out))
        return out

    def cell_faces(self, cell, q):
        """The reconstructed face values of `cell` on its six sides for the field q (one per cell)."""
        out = np.zeros(6)
        qq = np.ascontiguousarray(q, dtype=np.float64)
        lib().orc_cell_faces(self.h, int(cell), _p(qq), _p(out))
        return out

    def face_nsf(self, W, cell, side):
        """orc_face_nsf: the synthetic solve's NSF stress (xx yy zz xy xz yz) and heat fluxes
        q_t, q_r at the face of `cell` on `side` for the conservative state W [cell][6]."""
        out = np.zeros(12)
        Wc = np.ascontiguousarray(W, dtype=np.float64)
        self._rc(lib().orc_face_nsf(self.h, _p(Wc), int(cell), int(side), _p(out)), "orc_face_nsf")
        return out

    def cell_gradient(self, cell, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        g = np.empty(3)
        lib().orc_cell_gradient(self.h, cell, _p(q), _p(g))
        return g

    def cell_limiter(self, cell, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        return lib().orc_cell_limiter(self.h, cell, _p(q))

    def geometry(self):
        vol = np.empty(self.nc)
        xc = np.empty((self.nc, 3))
        S = np.empty((self.nc, 6, 3))
        xf = np.empty((self.nc, 6, 3))
        lib().orc_get_geometry(self.h, _p(vol), _p(xc), _p(S), _p(xf))
        return vol, xc, S, xf


def tau(p, rho, Tt):
    g = gas_struct(p)
    return lib().orc_tau(C.byref(g), rho, Tt)


def conductivity(p, mu):
    g = gas_struct(p)
    kt, kr = C.c_double(), C.c_double()
    lib().orc_conductivity(C.byref(g), mu, C.byref(kt), C.byref(kr))
    return kt.value, kr.value


def reference(p, state12, xi):
    g = gas_struct(p)
    st = np.ascontiguousarray(state12, dtype=np.float64)
    x = np.ascontiguousarray(xi, dtype=np.float64)
    g0, g1 = C.c_double(), C.c_double()
    lib().orc_reference(C.byref(g), _p(st), _p(x), C.byref(g0), C.byref(g1))
    return g0.value, g1.value


def venkat_face(dm, d2, eps2):
    return lib().orc_venkat_face(dm, d2, eps2)

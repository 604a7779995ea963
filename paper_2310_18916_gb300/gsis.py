"""Thin Python binding of the C ABI in include/gsis.h (argument marshalling only).

Every step of the solver runs in libgsis.so; PyTorch supplies the CUDA stream and, through the
allocator callback, device memory from its caching allocator.  There is no CPU fallback: if the
library or a GPU is missing, constructing a Solver raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgsis.so")

D = C.POINTER(C.c_double)
GSIS_OK, GSIS_E_TIMEOUT, GSIS_E_NOT_CONVERGED, GSIS_E_UNSUPPORTED = 0, -5, -6, -7
F64, F32, BF16 = 0, 1, 2
PRECISIONS = {"f64": F64, "f32": F32, "bf16": BF16}
MODE_GSIS, MODE_DVM = 0, 1
F_W, F_HALF, F_HOT = 1, 2, 4
ERRORS = {-1: "GSIS_E_INVALID", -2: "GSIS_E_OOM", -3: "GSIS_E_CUDA", -4: "GSIS_E_DIVERGED", -5: "GSIS_E_TIMEOUT",
          -6: "GSIS_E_NOT_CONVERGED", -7: "GSIS_E_UNSUPPORTED"}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)
ALLREDUCE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Mesh(C.Structure):
    _fields_ = [("ni", C.c_int), ("nj", C.c_int), ("nk", C.c_int), ("nodes", D), ("bc", C.c_int * 6),
                ("wall_u", (C.c_double * 3) * 6), ("wall_T", C.c_double * 6), ("ncells", C.c_int), ("nnodes", C.c_int),
                ("unodes", D), ("cells", C.POINTER(C.c_int)), ("face_patch", C.POINTER(C.c_int))]


class Vgrid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("x", D * 3), ("w", D * 3), ("npoints", C.c_int), ("points", D)]


class Gas(C.Structure):
    _fields_ = [("model", C.c_int), ("omega", C.c_double), ("d_r", C.c_double), ("Z_r", C.c_double),
                ("A", C.c_double * 4)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("mode", C.c_int), ("n_sweeps", C.c_int), ("macro_steps", C.c_int),
                ("macro_sweeps", C.c_int), ("macro_cfl", C.c_double), ("macro_tol", C.c_double),
                ("kin_inv_dt", C.c_double), ("venkat_K", C.c_double), ("kinetic_presteps", C.c_int),
                ("init_W", D), ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("macro_sms", C.c_int), ("shard_count", C.c_int),
                ("shard_index", C.c_int), ("allreduce", ALLREDUCE_FN), ("allreduce_ctx", C.c_void_p),
                ("kinetic_ring", C.c_int), ("euler_presteps", C.c_int),
                ("wall_flux", C.c_int), ("positive_faces", C.c_int),
                ("relax", C.c_double), ("visc_jump", C.c_double), ("capture_graphs", C.c_int)]


_lib = None
SYMBOLS = ("gsis_default_options", "gsis_footprint_bytes", "gsis_create", "gsis_iterate", "gsis_step_async",
           "gsis_step_wait", "gsis_moments",
           "gsis_residual", "gsis_nwall", "gsis_wall", "gsis_wall_loads", "gsis_kinetic_flux_sum", "gsis_get_f", "gsis_set_f", "gsis_stats",
           "gsis_graphs",
           "gsis_destroy", "gsis_last_error", "gsis_profile", "gsis_vdf_moments_noalloc", "gsis_selftest_wait_timeout")


def load(path: str = LIB_PATH):
    """Load libgsis.so and declare its entry points (no GPU needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run __graft_entry__.build() first")
    L = C.CDLL(path)
    P = C.c_void_p
    L.gsis_default_options.argtypes = [C.POINTER(Options)]
    L.gsis_footprint_bytes.argtypes = [C.POINTER(Mesh), C.POINTER(Vgrid), C.POINTER(Gas), C.POINTER(Options),
                                       C.POINTER(C.c_size_t)]
    L.gsis_create.argtypes = [C.POINTER(Mesh), C.POINTER(Vgrid), C.POINTER(Gas), C.c_double, C.c_double,
                              C.POINTER(Options), C.POINTER(P)]
    L.gsis_iterate.argtypes = [P, C.c_int, C.c_double, C.POINTER(C.c_int), D]
    L.gsis_step_async.argtypes = [P]
    L.gsis_step_wait.argtypes = [P, D]
    L.gsis_moments.argtypes = [P, C.c_uint, D, C.c_size_t]
    L.gsis_residual.argtypes = [P, D, C.c_int]
    L.gsis_nwall.argtypes = [P]
    L.gsis_wall.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int), D, D]
    L.gsis_wall_loads.argtypes = [P, C.c_uint, D, C.c_double, C.c_double, C.c_double, D]
    L.gsis_kinetic_flux_sum.argtypes = [P, D, C.c_size_t]
    L.gsis_get_f.argtypes = [P, D, D]
    L.gsis_set_f.argtypes = [P, D, D]
    L.gsis_stats.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.gsis_graphs.argtypes = [P]
    L.gsis_profile.argtypes = [P, C.c_int, C.c_int, D, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.gsis_vdf_moments_noalloc.argtypes = [P, P, C.c_int, C.c_int, P, P]
    L.gsis_destroy.argtypes = [P]
    L.gsis_last_error.argtypes = [P]
    L.gsis_last_error.restype = C.c_char_p
    L.gsis_selftest_wait_timeout.argtypes = [C.c_int, C.POINTER(C.c_int)]
    _lib = L
    return L


def _p(a):
    return a.ctypes.data_as(D)


class GsisError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def build_structs(problem, keep):
    """Marshal a workloads.Problem into the ABI's mesh, velocity grid and gas structs."""
    nodes = np.ascontiguousarray(problem.nodes, dtype=np.float64)
    keep.append(nodes)
    m = Mesh()
    m.ni, m.nj, m.nk = problem.ni, problem.nj, problem.nk
    m.nodes = _p(nodes)
    if getattr(problem, "ucells", None) is not None:
        un = np.ascontiguousarray(problem.unodes, dtype=np.float64)
        uc = np.ascontiguousarray(problem.ucells, dtype=np.int32)
        up = np.ascontiguousarray(problem.upatch, dtype=np.int32)
        keep += [un, uc, up]
        m.ncells, m.nnodes = len(uc), len(un)
        m.unodes = _p(un)
        m.cells = uc.ctypes.data_as(C.POINTER(C.c_int))
        m.face_patch = up.ctypes.data_as(C.POINTER(C.c_int))
    for s in range(6):
        m.bc[s] = int(problem.bc[s])
        m.wall_T[s] = float(problem.wall_T[s])
        for d in range(3):
            m.wall_u[s][d] = float(problem.wall_u[s][d])
    vg = Vgrid()
    for a, (x, w) in enumerate(((problem.vx, problem.wx), (problem.vy, problem.wy), (problem.vz, problem.wz))):
        x = np.ascontiguousarray(x, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        keep += [x, w]
        vg.n[a] = len(x)
        vg.x[a] = _p(x)
        vg.w[a] = _p(w)
    if getattr(problem, "vpoints", None) is not None:
        pts = np.ascontiguousarray(problem.vpoints, dtype=np.float64)
        keep.append(pts)
        vg.npoints = len(pts)
        vg.points = _p(pts)
    g = Gas()
    g.model, g.omega, g.d_r, g.Z_r = problem.model, problem.omega, problem.d_r, problem.Z_r
    for k in range(4):
        g.A[k] = problem.A[k]
    return m, vg, g


class Solver:
    """GSIS solver on one GPU for a workloads.Problem.

    precision: "f32", "f64" or "bf16" (VDF storage; kinetic arithmetic is FP32 for f32 and bf16,
    FP64 for f64; the synthetic solve is FP64).
    mode: "gsis" or "dvm".  Other keyword arguments map onto gsis_options.
    shard: (index, count) of a velocity-sharded solve, with allreduce(ptr, count, stream_ptr) the
    sum-all-reduce of count FP64 values at device pointer ptr (see sharding.py).
    """

    def __init__(self, problem, precision="f32", mode="gsis", init_W=None, torch_memory=True, shard=None,
                 allreduce=None, **opts):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the GSIS library needs a CUDA GPU")
        L = load()
        self.problem = problem
        self._keep = []
        m, vg, g = build_structs(problem, self._keep)
        o = Options()
        L.gsis_default_options(C.byref(o))
        o.precision = PRECISIONS[precision]
        o.mode = MODE_GSIS if mode == "gsis" else MODE_DVM
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        if shard is not None:
            if allreduce is None:
                raise TypeError("a sharded solve needs allreduce")
            o.shard_index, o.shard_count = int(shard[0]), int(shard[1])

            def _allreduce(ptr, count, stream, ctx):
                try:
                    allreduce(int(ptr), int(count), int(stream or 0))
                    return 0
                except Exception:  # noqa: BLE001 - reported to the library as a failed exchange
                    import traceback
                    traceback.print_exc()
                    return 1

            self._allreduce_cb = ALLREDUCE_FN(_allreduce)
            o.allreduce = self._allreduce_cb
        W0 = problem.W0 if init_W is None else init_W
        if W0 is not None:
            W0 = np.ascontiguousarray(W0, dtype=np.float64)
            self._keep.append(W0)
            o.init_W = _p(W0)
        self.stream = torch.cuda.current_stream()
        o.stream = C.c_void_p(self.stream.cuda_stream)
        if torch_memory:
            dev = torch.cuda.current_device()
            sptr = self.stream.cuda_stream

            def _alloc(nbytes, stream, ctx):
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, sptr)

            def _free(ptr, stream, ctx):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
            o.alloc = self._alloc_cb
            o.free = self._free_cb
        self.options = o
        h = C.c_void_p()
        rc = L.gsis_create(C.byref(m), C.byref(vg), C.byref(g), float(problem.Kn), float(problem.Ma), C.byref(o),
                           C.byref(h))
        if rc != 0:
            raise GsisError(rc, L.gsis_last_error(None).decode())
        self.h = h
        self.nc = problem.ncells
        self.nv = problem.nvel
        self.nwall = L.gsis_nwall(h)

    def _check(self, rc, ok=(GSIS_OK,)):
        if rc not in ok:
            raise GsisError(rc, load().gsis_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            load().gsis_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def iterate(self, max_outer=1, tol=0.0):
        done, eps = C.c_int(), C.c_double()
        rc = load().gsis_iterate(self.h, max_outer, tol, C.byref(done), C.byref(eps))
        self._check(rc, (GSIS_OK, GSIS_E_NOT_CONVERGED))
        return done.value, eps.value, rc == GSIS_OK

    def step(self):
        return self.iterate(1, 0.0)[1]

    def step_async(self):
        """Enqueue one outer step on the solver's stream; step_wait() returns its eps."""
        self._check(load().gsis_step_async(self.h))

    def step_wait(self):
        eps = C.c_double()
        self._check(load().gsis_step_wait(self.h, C.byref(eps)))
        return eps.value

    def moments(self, mask=F_W):
        per = (6 if mask & F_W else 0) + (18 if mask & F_HALF else 0) + (12 if mask & F_HOT else 0)
        out = np.empty((self.nc, per))
        self._check(load().gsis_moments(self.h, mask, _p(out), out.size))
        return out

    def W(self):
        return self.moments(F_W)

    def half_moments(self):
        return self.moments(F_HALF)

    def hot(self):
        return self.moments(F_HOT)

    def residual(self):
        out = np.empty(4)
        self._check(load().gsis_residual(self.h, _p(out), 4))
        return out

    def wall(self):
        n = self.nwall
        cell = np.empty(n, dtype=np.int32)
        side = np.empty(n, dtype=np.int32)
        rw = np.empty(n)
        fl = np.empty((n, 6))
        self._check(load().gsis_wall(self.h, cell.ctypes.data_as(C.POINTER(C.c_int)),
                                     side.ctypes.data_as(C.POINTER(C.c_int)), _p(rw), _p(fl)))
        return cell, side, rw, fl

    def wall_loads(self, sides, direction, rho_ref, U_ref, A_ref):
        """Force (3), energy flux, C_D, C_H on the walls of the given sides (0 -x .. 5 +z)."""
        mask = 0
        for sd in sides:
            mask |= 1 << int(sd)
        d = np.ascontiguousarray(direction, dtype=np.float64)
        out = np.empty(6)
        self._check(load().gsis_wall_loads(self.h, mask, _p(d), float(rho_ref), float(U_ref), float(A_ref), _p(out)))
        return out

    def kinetic_flux_sum(self):
        out = np.empty((self.nc, 6))
        self._check(load().gsis_kinetic_flux_sum(self.h, _p(out), out.size))
        return out

    def get_f(self, both=False):
        """f0 [cell][v]; with both=True (Rykov) the pair (f0, f1)."""
        f0 = np.empty((self.nc, self.nv))
        f1 = np.empty((self.nc, self.nv)) if both else None
        self._check(load().gsis_get_f(self.h, _p(f0), _p(f1) if both else None))
        return (f0, f1) if both else f0

    def set_f(self, f0, f1=None):
        f0 = np.ascontiguousarray(f0, dtype=np.float64)
        f1 = None if f1 is None else np.ascontiguousarray(f1, dtype=np.float64)
        self._check(load().gsis_set_f(self.h, _p(f0), None if f1 is None else _p(f1)))

    def profile(self, enable=True, reset=False):
        """Per-phase device milliseconds (wall, kinetic, reduce, synthetic, state), steps, launches."""
        ms = np.zeros(5)
        st, la = C.c_int(), C.c_int()
        self._check(load().gsis_profile(self.h, int(enable), int(reset), _p(ms), 5, C.byref(st), C.byref(la)))
        return ms, st.value, la.value

    def stats(self):
        a, b = C.c_int(), C.c_int()
        self._check(load().gsis_stats(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def graphs(self):
        """Captured outer-step graphs held (-1: a capture failed, steps launch directly)."""
        return load().gsis_graphs(self.h)


_NO_EXCHANGE = ALLREDUCE_FN(lambda ptr, count, stream, ctx: 1)  # footprints never exchange


def selftest_wait_timeout(which):
    """Run a bounded device wait that cannot complete (0: the grid barrier of the synthetic
    solve, 1: the kinetic kernel's mbarrier wait) and return the device error status it raised
    (GSIS_E_TIMEOUT when the wait ran out as designed)."""
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("the GSIS library needs a CUDA GPU")
    st = C.c_int()
    rc = load().gsis_selftest_wait_timeout(int(which), C.byref(st))
    if rc != GSIS_OK:
        raise GsisError(rc, "self-test launch failed")
    return st.value


def footprint_bytes(problem, precision="f32", shard=None, **opts):
    """Device bytes a solver of this problem holds (shard: (index, count) of a sharded solve;
    other keyword arguments map onto gsis_options)."""
    L = load()
    keep = []
    m, vg, g = build_structs(problem, keep)
    o = Options()
    L.gsis_default_options(C.byref(o))
    o.precision = PRECISIONS[precision]
    for k, v in opts.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    if shard is not None:
        o.shard_index, o.shard_count = int(shard[0]), int(shard[1])
        o.allreduce = _NO_EXCHANGE
    out = C.c_size_t()
    rc = L.gsis_footprint_bytes(C.byref(m), C.byref(vg), C.byref(g), C.byref(o), C.byref(out))
    if rc != 0:
        raise GsisError(rc, "footprint")
    return out.value

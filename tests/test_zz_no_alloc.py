"""The allocation-free moments entry point (for callers that cannot allocate device memory)
against the solver's own moments of the same VDF, on two calls in a row.

Collected last on purpose: if it fails, a run that stops at the first failure has already run
every other test.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_common import scaled_close

pytestmark = pytest.mark.gpu


def _velocity_table(p):
    X, Y, Z = np.meshgrid(p.vx, p.vy, p.vz, indexing="ij")
    Wt = p.wx[:, None, None] * p.wy[None, :, None] * p.wz[None, None, :]
    flat = lambda a: a.transpose(2, 1, 0).ravel()   # v = ix + nx (iy + ny iz)
    return np.stack([flat(X), flat(Y), flat(Z), flat(Wt)], axis=1).astype(np.float32)


def test_noalloc_moments_match_the_solver_on_two_calls():
    import torch

    from paper_2310_18916_gb300 import gsis
    from paper_2310_18916_gb300 import workloads as wl

    p = wl.cavity(n=10, nv=16, Kn=0.1)
    W = wl.perturbed_state(p, seed=11, amp=0.05)
    f0, _ = wl.random_vdf(p, seed=12, amp=0.2, W=W)
    f32 = f0.astype(np.float32)
    # existing entry points: the solver stores f in FP32 and reports its moments
    s = gsis.Solver(p, precision="f32", kinetic_presteps=0)
    s.set_f(f32.astype(np.float64))
    ref = s.half_moments()
    s.close()

    L = gsis.load()
    f_dev = torch.from_numpy(f32).cuda()
    vel_dev = torch.from_numpy(_velocity_table(p)).cuda()
    out = torch.empty((p.ncells, 18), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out.fill_(float("nan"))
        rc = L.gsis_vdf_moments_noalloc(C.c_void_p(f_dev.data_ptr()), C.c_void_p(vel_dev.data_ptr()), p.ncells,
                                        p.nvel, C.c_void_p(out.data_ptr()), C.c_void_p(stream))
        assert rc == 0, f"call {call}: rc {rc}"
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        scaled_close(got[:, :12], ref[:, :12], 2e-5, f"moments, call {call}")
        scaled_close(got[:, 12:15], ref[:, 12:15], 2e-4, f"heat flux, call {call}", vector=True)


def _fast_stream(ncells, nv, vmax, seed):
    """Seeded VDFs of a Ma-4 stream (u = 4 sqrt(5/6) along x, T = 1) with a smooth positive
    non-equilibrium modulation per cell, and their moments by definition in FP64 (about the mean
    velocity, Eq. getmoment) from the same FP32 values."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nv) + 0.5) * (2 * vmax / nv) - vmax
    w = np.full(nv, 2 * vmax / nv)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    flat = lambda a: a.transpose(2, 1, 0).ravel()
    xi = np.stack([flat(X), flat(Y), flat(Z)], 1)
    Wt = flat(w[:, None, None] * w[None, :, None] * w[None, None, :])
    vel = np.concatenate([xi, Wt[:, None]], 1).astype(np.float32)
    U = 4.0 * np.sqrt(5.0 / 6.0)
    f = np.empty((ncells, len(Wt)), dtype=np.float32)
    for i in range(ncells):
        rho, T = rng.uniform(0.8, 1.2), rng.uniform(0.8, 1.2)
        u = np.array([U, 0.0, 0.0]) + rng.uniform(-0.1, 0.1, 3)
        c = xi - u
        c2 = (c * c).sum(1)
        a = rng.uniform(-0.05, 0.05, 3)
        f[i] = rho * (np.pi * T) ** -1.5 * np.exp(-c2 / T) * (1 + (c @ a) * (c2 / T - 2.5) * np.exp(-c2 / (4 * T)))
    xd, wd = vel[:, :3].astype(np.float64), vel[:, 3].astype(np.float64)
    ref = np.zeros((ncells, 18))
    for i in range(ncells):
        fw = wd * f[i].astype(np.float64)
        rho = fw.sum()
        u = (fw[:, None] * xd).sum(0) / rho
        c = xd - u
        c2 = (c * c).sum(1)
        P = (fw[:, None, None] * c[:, :, None] * c[:, None, :]).sum(0)
        tr = np.trace(P) / 3
        ref[i, 0], ref[i, 1:4] = rho, u
        ref[i, 4] = ref[i, 5] = 2 * np.trace(P) / (3 * rho)
        ref[i, 6:12] = [P[0, 0] - tr, P[1, 1] - tr, P[2, 2] - tr, P[0, 1], P[0, 2], P[1, 2]]
        ref[i, 12:15] = (fw[:, None] * (0.5 * c2)[:, None] * c).sum(0)
    return f, vel, ref


@pytest.mark.parametrize("ncells", [1, 5])
def test_noalloc_moments_of_a_mach4_stream_on_a_48_cubed_grid(ncells):
    """A fast stream on the 48^3 velocity grid (110592 velocities; a single cell needs many
    velocity chunks): the moments about the mean velocity keep FP32 accuracy although |u| is
    3.7 times the thermal speed (stress within 2e-5 of the pressure, heat flux within 2e-4 of
    rho T^(3/2)), on two calls in a row."""
    import torch

    from paper_2310_18916_gb300 import gsis

    f, vel, ref = _fast_stream(ncells, 48, 12.0, seed=21 + ncells)
    L = gsis.load()
    f_dev = torch.from_numpy(f).cuda()
    vel_dev = torch.from_numpy(vel).cuda()
    out = torch.empty((ncells, 18), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    p = 0.5 * ref[:, 0] * ref[:, 4]
    qs = ref[:, 0] * ref[:, 4] ** 1.5
    for call in range(2):
        out.fill_(float("nan"))
        rc = L.gsis_vdf_moments_noalloc(C.c_void_p(f_dev.data_ptr()), C.c_void_p(vel_dev.data_ptr()), ncells,
                                        f.shape[1], C.c_void_p(out.data_ptr()), C.c_void_p(stream))
        assert rc == 0, f"call {call}: rc {rc}"
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got[:, 0] / ref[:, 0] - 1).max() < 2e-6
        assert np.abs(got[:, 1:4] - ref[:, 1:4]).max() < 2e-6 * np.abs(ref[:, 1:4]).max()
        assert np.abs(got[:, 4] / ref[:, 4] - 1).max() < 2e-5
        assert (np.abs(got[:, 6:12] - ref[:, 6:12]) / p[:, None]).max() < 2e-5
        assert (np.abs(got[:, 12:15] - ref[:, 12:15]) / qs[:, None]).max() < 2e-4


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2310_18916_gb300 import gsis

    L = gsis.load()
    one = C.c_void_p(16)   # never dereferenced: the size check comes first
    assert L.gsis_vdf_moments_noalloc(one, one, 87382, 8, one, None) == -1
    assert b"87381" in L.gsis_last_error(None)

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


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2310_18916_gb300 import gsis

    L = gsis.load()
    one = C.c_void_p(1)   # never dereferenced: the size check comes first
    assert L.gsis_vdf_moments_noalloc(one, one, 80660, 8, one, None) == -1

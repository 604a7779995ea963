"""BF16 VDF storage (FP32 kinetic arithmetic, FP32 compensated moments, FP64 synthetic solve).

BF16 keeps 8 significant bits: a stored value is within u = 2^-8 of the FP32 value it rounds
(round to nearest even), relative.  A moment sum_v w phi f therefore moves by at most u of
sum_v w |phi| f, so per-step states agree with the FP32-storage path to a few u of their scale
(bound 4u for three steps; the iteration is contractive).  Converged density and temperature
are held to 1e-3 relative L2 of the FP64 oracle, the accuracy required of BF16 storage.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8


def _rel_l2(a, b, vol):
    return np.sqrt(((a - b) ** 2 * vol).sum() / (b ** 2 * vol).sum())


def test_bf16_steps_track_fp32_storage():
    p = wl.cavity(n=16, nv=16, Kn=0.1, lid=0.16)
    a = gsis.Solver(p, precision="bf16", mode="gsis", kinetic_presteps=0, macro_steps=100)
    b = gsis.Solver(p, precision="f32", mode="gsis", kinetic_presteps=0, macro_steps=100)
    for it in range(3):
        a.step()
        b.step()
        Wa, Wb = a.W(), b.W()
        scale = np.maximum(np.abs(Wb).max(axis=0), 1e-3 * np.abs(Wb).max())
        err = (np.abs(Wa - Wb) / scale).max()
        assert err < 4 * U_BF16, f"step {it}: {err:.3e}"
    # the storage is really BF16: the two paths differ by more than FP32 round-off
    assert err > 1e-6


def test_cavity_bf16_converged_within_bf16_tolerance():
    """BF16 storage leaves eps a floor near its round-off; the GPU runs until eps < 1e-4 (or 150
    steps) and is compared with the oracle converged to 1e-6."""
    p = wl.cavity(n=24, nv=16, Kn=0.1, lid=0.16)
    g = gsis.Solver(p, precision="bf16", mode="gsis")
    done, eps, ok = g.iterate(150, 1e-4)
    o = Oracle(p, mode=0)
    o.presteps(10)
    ho = o.run(150, 1e-6)
    assert ho[-1] < 1e-6
    vol = o.geometry()[0]
    Wg, Wo = g.W(), o.W()
    e_rho = _rel_l2(Wg[:, 0], Wo[:, 0], vol)
    e_T = _rel_l2(Wg[:, 4], Wo[:, 4], vol)
    print(f"bf16 cavity 24^2: {done} steps, eps {eps:.2e}, rel-L2 rho {e_rho:.2e}, E {e_T:.2e}")
    assert e_rho < 1e-3
    assert e_T < 1e-3
    assert np.abs(Wg[:, 1:3] - Wo[:, 1:3]).max() < 1e-2 * np.abs(Wo[:, 1:3]).max()


@pytest.mark.parametrize("rykov", [False, True])
def test_cavity_bf16_long_run_at_64_squared_against_the_gpu_fp64_path(rykov):
    """A long BF16 run on a larger cavity (64^2 cells, 24^3 velocities, Kn 0.05), Shakhov and
    Rykov: until eps < 1e-4 or 200 steps, against the plain FP64 GPU path converged to 1e-8 on
    the same inputs (the FP64 path itself matches the oracle to 1e-10 per step in the parity
    tests).  Density and temperature within 1e-3 relative L2, velocity within 1 % of its scale."""
    p = wl.cavity(n=64, nv=24, Kn=0.05, lid=0.16)
    if rykov:
        p = wl.as_rykov(p)
    ref = gsis.Solver(p, precision="f64", mode="gsis")
    _, eps_ref, _ = ref.iterate(200, 1e-8)
    assert eps_ref < 1e-8
    Wr = ref.W()
    ref.close()
    g = gsis.Solver(p, precision="bf16", mode="gsis")
    done, eps, _ = g.iterate(200, 1e-4)
    Wg = g.W()
    g.close()
    vol = np.full(p.ncells, 1.0 / p.ncells)
    e_rho = _rel_l2(Wg[:, 0], Wr[:, 0], vol)
    e_T = _rel_l2(Wg[:, 4], Wr[:, 4], vol)
    print(f"bf16 cavity 64^2 {'Rykov' if rykov else 'Shakhov'}: {done} steps, eps {eps:.2e}, "
          f"rel-L2 rho {e_rho:.2e}, T {e_T:.2e}")
    assert e_rho < 1e-3 and e_T < 1e-3
    assert np.abs(Wg[:, 1:3] - Wr[:, 1:3]).max() < 1e-2 * np.abs(Wr[:, 1:3]).max()

"""Velocity-sharded solves on one GPU (K logical shards, one thread and stream each, exchanging
through the in-process all-reduce): every shard holds the same state after each step, and it
matches the unsharded solve to round-off (partial sums are added in another order)."""
import numpy as np
import pytest

from gpu_common import scaled_close
from paper_2310_18916_gb300 import gsis, sharding
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

OPTS = dict(macro_steps=60, macro_tol=0.0, kinetic_presteps=2)


@pytest.mark.parametrize("k,precision,model,tol", [(2, "f64", "shakhov", 1e-11), (3, "f64", "shakhov", 1e-11),
                                                  (2, "f32", "shakhov", 2e-6), (2, "f64", "rykov", 1e-11)])
def test_local_shards_match_the_unsharded_solve(k, precision, model, tol):
    p = wl.cavity(n=10, nv=12, Kn=0.1, lid=0.2)
    if model == "rykov":
        p = wl.as_rykov(p)
    hist = sharding.run_local_shards(p, k, steps=3, precision=precision, mode="gsis", **OPTS)
    ref = gsis.Solver(p, precision=precision, mode="gsis", **OPTS)
    for it in range(3):
        ref.step()
        for i in range(1, k):
            np.testing.assert_array_equal(hist[i][it], hist[0][it])  # replicated identically
        scaled_close(hist[0][it], ref.W(), tol, f"{k} shards {precision} {model}, step {it}")


@pytest.mark.parametrize("mode", ["dvm", "gsis"])
def test_local_shards_on_a_cylinder_ogrid(mode):
    """Velocity shards on a general mesh: the wall densities divide each shard's numerator by the
    re-emission flux over every velocity, the kinetic face-flux sums are all-reduced before the
    synthetic solve."""
    p = wl.cylinder(n_r=5, n_theta=10, nv=12, R=0.5, R_out=3.0, Ma=0.5, Kn=0.2)
    opts = dict(macro_steps=40, macro_tol=0.0, kinetic_presteps=0, n_sweeps=2)
    hist = sharding.run_local_shards(p, 2, steps=3, precision="f64", mode=mode, **opts)
    ref = gsis.Solver(p, precision="f64", mode=mode, **opts)
    for it in range(3):
        ref.step()
        np.testing.assert_array_equal(hist[1][it], hist[0][it])
        scaled_close(hist[0][it], ref.W(), 1e-11, f"2 shards on a cylinder ({mode}), step {it}")

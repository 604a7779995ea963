"""Helpers shared by the GPU tests: build the CUDA solver and the oracle on the same inputs."""
import numpy as np

from oracle.oracle import Oracle
from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl


def pair(p, precision="f64", mode="gsis", W0=None, **opts):
    """(GPU solver, oracle) with identical options; no presteps unless asked."""
    presteps = opts.pop("kinetic_presteps", 0)
    macro_steps = opts.pop("macro_steps", 300)
    macro_tol = opts.pop("macro_tol", 0.0)
    g = gsis.Solver(p, precision=precision, mode=mode, init_W=W0, kinetic_presteps=presteps,
                    macro_steps=macro_steps, macro_tol=macro_tol, **opts)
    o = Oracle(p, W0=W0, mode=0 if mode == "gsis" else 1, macro_steps=macro_steps, macro_tol=macro_tol)
    if presteps:
        o.presteps(presteps)
    return g, o


def scaled_close(a, b, rel, what, vector=False):
    """Column-wise |a - b| <= rel * max(|b| over cells, floor) with a floor for near-zero fields;
    vector=True scales every column by the largest column (components of one vector)."""
    a = np.asarray(a)
    b = np.asarray(b)
    scale = np.maximum(np.abs(b).max(axis=0), 1e-3 * np.abs(b).max())
    if vector:
        scale = np.full_like(scale, np.abs(b).max())
    err = (np.abs(a - b) / scale).max(axis=0)
    assert (err <= rel).all(), f"{what}: worst column error {err.max():.3e} (limit {rel:.1e}) per column {err}"
    return err.max()

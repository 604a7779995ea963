"""The C-ABI library loads and exports every entry point include/gsis.h declares (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gsis.h")).read()
    decl = re.findall(r"^(?:int|void|const char \*)\s*(gsis_[a-z_]+)\s*\(", src, flags=re.M)
    return sorted(set(decl))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_18916_gb300 import build as B
    path = B.build()
    from paper_2310_18916_gb300 import gsis
    return gsis.load(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("gsis_create", "gsis_iterate", "gsis_moments", "gsis_residual", "gsis_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2310_18916_gb300 import gsis
    out = subprocess.run(["nm", "-D", "--defined-only", gsis.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gsis_[a-z_]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)


def test_binding_declares_every_symbol():
    from paper_2310_18916_gb300 import gsis
    assert sorted(gsis.SYMBOLS) == _declared()


def test_default_options_and_footprint_without_gpu(lib):
    from paper_2310_18916_gb300 import gsis
    from paper_2310_18916_gb300 import workloads as wl
    import ctypes as C
    o = gsis.Options()
    lib.gsis_default_options(C.byref(o))
    assert o.precision == gsis.F32 and o.macro_steps == 300 and o.n_sweeps == 1 and o.kinetic_presteps == 10
    # footprint of the 128^2 x 32^3 cavity: f (4 B/point) dominates
    b = gsis.footprint_bytes(wl.cavity(n=128, nv=32), "f32")
    assert 4 * 128 * 128 * 32 ** 3 < b < 8 * 128 * 128 * 32 ** 3
    # BF16 storage halves the VDF: the footprints differ by 2 B per stored point
    pts = 128 * 128 * 32 ** 3
    assert b - gsis.footprint_bytes(wl.cavity(n=128, nv=32), "bf16") == 2 * pts

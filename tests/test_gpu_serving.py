"""Serving on the GPU: several steady solves admitted over time run concurrently on their own
streams; each result is identical to the same request served alone (same SM share)."""
import numpy as np
import pytest

from paper_2310_18916_gb300 import serving
from paper_2310_18916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_results_alone_and_in_the_mix_are_identical():
    rng = np.random.default_rng(3)
    probs = [wl.serving_cavity(rng, sizes=(16, 24), nvs=(12, 16)) for _ in range(5)]
    reqs = [serving.Request(i, p, arrival=0.02 * i, tol=1e-4, max_steps=40) for i, p in enumerate(probs)]
    budget = 8 << 30
    mix = serving.Server(budget, slots=3).run(reqs)
    assert all(r is not None for r in mix)
    assert sum(r.converged for r in mix) >= 4
    for r in reqs:
        alone = serving.Server(budget, slots=3).run([serving.Request(r.rid, r.problem, 0.0, r.tol, r.max_steps)])[0]
        m = mix[r.rid]
        assert alone.steps == m.steps
        assert alone.eps == m.eps
        assert np.array_equal(alone.W, m.W), f"request {r.rid}: max diff {np.abs(alone.W - m.W).max()}"


def test_admission_respects_the_memory_budget():
    rng = np.random.default_rng(5)
    probs = [wl.serving_cavity(rng, sizes=(16,), nvs=(12,)) for _ in range(3)]
    from paper_2310_18916_gb300 import gsis
    need = max(gsis.footprint_bytes(p, "f32") for p in probs)
    # room for one solve at a time: they run one after another and still all finish
    reqs = [serving.Request(i, p, 0.0, tol=1e-3, max_steps=20) for i, p in enumerate(probs)]
    res = serving.Server(int(1.5 * need), slots=3).run(reqs)
    spans = sorted((r.admitted, r.finished) for r in res)
    for (a0, f0), (a1, f1) in zip(spans, spans[1:]):
        assert a1 >= f0 - 1e-9


def test_mixed_stream_with_cylinders_and_kinetic_iteration_requests():
    """Cavities and cylinder O-grids in one stream, GSIS and plain kinetic-iteration requests side
    by side (each with its own solver options): every request finishes and gives the same result
    as when served alone."""
    rng = np.random.default_rng(0)
    drawn = [wl.serving_request(rng, sizes=(8, 12), nvs=(12,), kn=(0.05, 0.6), cavity_ma=(0.5, 3.0))
             for _ in range(6)]
    assert {o["mode"] for _, o in drawn} == {"gsis", "dvm"}
    assert any(p.name.startswith("cylinder") for p, _ in drawn) and any(p.name.startswith("cavity") for p, _ in drawn)
    reqs = [serving.Request(i, p, 0.01 * i, tol=1e-4, max_steps=40, opts=o) for i, (p, o) in enumerate(drawn)]
    budget = 8 << 30
    mix = serving.Server(budget, slots=3).run(reqs)
    assert all(r is not None for r in mix)
    for r in reqs:
        alone = serving.Server(budget, slots=3).run([serving.Request(r.rid, r.problem, 0.0, r.tol, r.max_steps,
                                                                     opts=r.opts)])[0]
        m = mix[r.rid]
        assert alone.steps == m.steps and alone.eps == m.eps
        assert np.array_equal(alone.W, m.W), f"request {r.rid} ({r.problem.name}, {r.opts})"

"""Scheduling logic of the serving loop on the CPU, with fake solvers and a fake clock:
first-in first-out admission by footprint and slots, rejection of requests larger than the
whole budget, results and latencies, percentiles."""
import numpy as np
import pytest

from paper_2310_18916_gb300 import serving


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeSolver:
    """eps halves every step; every step_wait advances the clock by dt."""

    log = []

    def __init__(self, problem, clock, dt):
        self.p, self.clock, self.dt, self.k = problem, clock, dt, 0
        self.pending = False
        FakeSolver.log.append(("create", problem["name"], clock()))

    def step_async(self):
        assert not self.pending
        self.pending = True

    def step_wait(self):
        assert self.pending
        self.pending = False
        self.k += 1
        self.clock.t += self.dt
        return 0.5 ** self.k

    def W(self):
        return np.full((2, 6), float(self.k))

    def close(self):
        FakeSolver.log.append(("close", self.p["name"], self.clock()))


def make_server(budget, slots, clock, dt=0.01):
    return serving.Server(budget, slots=slots, nsm=152,
                          make_solver=lambda p, prec, sms, st: FakeSolver(p, clock, dt),
                          footprint=lambda p, prec: p["bytes"], new_stream=lambda: None, clock=clock,
                          idle=lambda s: setattr(clock, "t", clock.t + max(s, 1e-3)))


def test_fifo_admission_by_footprint_and_slots():
    FakeSolver.log = []
    clock = FakeClock()
    reqs = [serving.Request(i, {"name": f"r{i}", "bytes": b}, a, tol=1.5 * 2 ** -5)
            for i, (b, a) in enumerate([(60, 0.0), (50, 0.0), (30, 0.0), (10, 0.5), (200, 0.6)])]
    srv = make_server(100, slots=2, clock=clock)
    assert srv.macro_sms == 76
    res = srv.run(reqs)
    # r0 (60) runs first; r1 (50) does not fit next to it and blocks r2 behind it (FIFO)
    creates = [name for kind, name, _ in FakeSolver.log if kind == "create"]
    assert creates == ["r0", "r1", "r2", "r3"]
    t = {name: tt for kind, name, tt in FakeSolver.log if kind == "create"}
    c = {name: tt for kind, name, tt in FakeSolver.log if kind == "close"}
    assert t["r1"] >= c["r0"]
    assert res[4] is None  # larger than the whole budget
    for r in res[:4]:
        assert r.converged and r.steps == 5 and r.eps == 2 ** -5
        assert r.latency >= r.steps * 0.01 - 1e-12
        assert r.admitted >= r.arrival
        assert (r.W == 5.0).all()


def test_a_stalled_eps_stops_at_the_precision_floor():
    class Flat(FakeSolver):
        def step_wait(self):
            super().step_wait()
            return 1e-3  # never improves after the first step
    clock = FakeClock()
    srv = serving.Server(10, slots=1, nsm=152, make_solver=lambda p, prec, sms, st: Flat(p, clock, 0.01),
                         footprint=lambda p, prec: 1, new_stream=lambda: None, clock=clock)
    res = srv.run([serving.Request(0, {"name": "f"}, 0.0, tol=1e-6, max_steps=100, stall_steps=7)])
    assert res[0].steps == 8 and res[0].floor and not res[0].converged
    assert serving.summary(res, clock.t)["at_precision_floor"] == 1


def test_idle_until_next_arrival_and_summary():
    FakeSolver.log = []
    clock = FakeClock()
    reqs = [serving.Request(0, {"name": "a", "bytes": 1}, 2.0, tol=0.3)]
    res = make_server(10, slots=4, clock=clock).run(reqs)
    assert res[0].admitted >= 2.0
    s = serving.summary(res, wall_seconds=clock.t)
    assert s["served"] == 1 and s["converged"] == 1
    assert s["p50_latency_s"] == pytest.approx(res[0].latency)


def test_percentile_matches_numpy():
    x = np.random.default_rng(1).exponential(1.0, 37)
    for q in (0, 50, 90, 99, 100):
        assert serving.percentile(x, q) == pytest.approx(np.percentile(x, q))


def test_poisson_requests_are_seeded():
    mk = lambda rng: {"n": int(rng.integers(10))}
    a = serving.poisson_requests(20, 2.0, 0, mk)
    b = serving.poisson_requests(20, 2.0, 0, mk)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert (gaps > 0).all() and abs(gaps.mean() - 2.0) < 1.2


def test_the_mixed_request_stream():
    """The serving mix: cavities and cylinders with equal odds, Kn log-uniform, lid Mach numbers up
    to 5 (up to 1.75 below Kn 0.05), subsonic cylinders below Kn 0.2 with two colour passes, GSIS
    below Kn 0.3 and the plain kinetic iteration above."""
    import numpy as np

    from paper_2310_18916_gb300 import workloads as wl

    reqs = serving.poisson_requests(300, 0.5, 7, lambda rng: wl.serving_request(rng))
    cyl = [r for r in reqs if r.problem.name.startswith("cylinder")]
    cav = [r for r in reqs if r.problem.name.startswith("cavity")]
    assert len(cyl) + len(cav) == 300 and 110 < len(cyl) < 190
    for r in reqs:
        assert 1e-3 <= r.problem.Kn <= 1.0
        assert r.opts["mode"] == ("gsis" if r.problem.Kn < 0.3 else "dvm")
    assert all(r.opts.get("n_sweeps") == 2 and r.problem.Kn <= 0.2 for r in cyl)
    assert all(0.1 <= r.problem.Ma <= 1.0 for r in cyl)
    assert all(r.problem.Ma <= (5.0 if r.problem.Kn >= 0.05 else 1.75) + 1e-9 for r in cav)
    assert max(r.problem.Ma for r in cav) > 3.0 and any(r.opts["mode"] == "dvm" for r in cav)
    assert all(r.problem.ncells in (32 * 64, 48 * 96, 64 * 128) for r in cyl)
    arrivals = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arrivals) > 0) and abs(np.diff(arrivals).mean() - 0.5) < 0.1


def test_a_failing_solve_leaves_with_its_error_and_the_others_finish():
    class Failing(FakeSolver):
        def step_wait(self):
            eps = super().step_wait()
            if self.p["name"] == "bad" and self.k == 3:
                raise RuntimeError("GSIS_E_DIVERGED: non-finite or non-positive density/temperature")
            return eps

    clock = FakeClock()
    srv = serving.Server(100, slots=2, nsm=152, make_solver=lambda p, prec, sms, st: Failing(p, clock, 0.01),
                         footprint=lambda p, prec: p["bytes"], new_stream=lambda: None, clock=clock,
                         idle=lambda s: setattr(clock, "t", clock.t + max(s, 1e-3)))
    reqs = [serving.Request(i, {"name": n, "bytes": 40}, 0.0, tol=2 ** -6) for i, n in enumerate(["a", "bad", "c"])]
    res = srv.run(reqs)
    assert "DIVERGED" in res[1].error and res[1].W is None and not res[1].converged and res[1].steps == 2
    assert res[0].converged and res[2].converged and not res[0].error
    s = serving.summary(res, 1.0)
    assert s["failed"] == 1 and s["served"] == 2 and s["converged"] == 2


def test_graphs_option_reaches_every_solver_unless_the_request_sets_it():
    FakeSolver.log = []
    clock = FakeClock()
    seen = []

    def make(p, prec, sms, st, **opts):
        seen.append((p["name"], opts.get("capture_graphs")))
        return FakeSolver(p, clock, 0.01)

    srv = serving.Server(100, slots=2, nsm=152, make_solver=make, footprint=lambda p, prec, **o: p["bytes"],
                         new_stream=lambda: None, clock=clock,
                         idle=lambda s: setattr(clock, "t", clock.t + max(s, 1e-3)), graphs=True)
    reqs = [serving.Request(0, {"name": "a", "bytes": 10}, 0.0, tol=1.5 * 2 ** -5),
            serving.Request(1, {"name": "b", "bytes": 10}, 0.0, tol=1.5 * 2 ** -5, opts={"capture_graphs": 0})]
    srv.run(reqs)
    assert sorted(seen) == [("a", 1), ("b", 0)]

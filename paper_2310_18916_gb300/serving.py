"""Serving loop for steady GSIS solves on one GPU: continuous batching of requests that arrive
over time (the serving form of the method's steady solves: each request is one run of
Algorithm 1 to eps < tol).

Requests are admitted first-in first-out when their device footprint (gsis_footprint_bytes)
fits in the memory budget next to the solves already running and a slot is free.  An admitted
solve keeps its VDF resident and advances one outer step per round on its own CUDA stream.
Each round enqueues the steps of all running solves before it waits for any, so their kernels
overlap on the device.  A solve leaves when eps < tol (or after max_steps) and frees its memory
and slot, and waiting requests are admitted at once.  A solve whose eps has not reached a new
minimum for stall_steps steps has hit the round-off floor of its storage precision (FP32 storage
puts it near 1e-6 for slow flows, where the velocity is small next to the thermal speed); it
leaves then, marked as stopped at its floor.

The FP64 synthetic solve of a step is one cooperative kernel whose blocks each hold a whole SM.
Every solve therefore gets a fixed share of the SMs (SM count // slots), so the cooperative
kernels of all slots fit on the GPU together.  The share also fixes the kernel's block count
and hence its reduction order: a request gives identical results alone and in the mix when
it runs with the same share.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    problem: object          # workloads.Problem
    arrival: float           # seconds after the start of the run
    tol: float = 1e-6
    max_steps: int = 400
    stall_steps: int = 20
    opts: dict = field(default_factory=dict)   # solver options of this request (mode, n_sweeps, ...)


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    eps: float
    converged: bool
    W: np.ndarray = field(repr=False, default=None)
    floor: bool = False      # stopped at the round-off floor (eps stalled above tol)
    error: str = ""          # the solver's error when the solve failed (its state then left no W)

    @property
    def latency(self) -> float:
        """Arrival to converged state, seconds."""
        return self.finished - self.arrival


def percentile(values, q):
    """q-th percentile (0..100) of values by linear interpolation between order statistics."""
    v = np.sort(np.asarray(values, dtype=float))
    if len(v) == 0:
        return float("nan")
    pos = (len(v) - 1) * q / 100.0
    lo = int(np.floor(pos))
    hi = min(lo + 1, len(v) - 1)
    return float(v[lo] + (v[hi] - v[lo]) * (pos - lo))


class _Running:
    def __init__(self, req, solver, stream, need, admitted):
        self.req, self.solver, self.stream, self.need, self.admitted = req, solver, stream, need, admitted
        self.steps, self.eps = 0, float("inf")
        self.best, self.since_best = float("inf"), 0


class Server:
    """Continuous-batching GSIS server on the current GPU.

    memory_budget: device bytes the running solves may hold together.
    slots: solves that run at the same time.
    precision: VDF storage of every solve ("f32", "bf16" or "f64").
    make_solver(problem, precision, macro_sms, stream, **opts) / footprint(problem, precision,
    **opts): the GPU solver and its footprint, opts the request's solver options; replaceable (the
    scheduling logic is tested with fakes).
    graphs: every solve runs its outer steps as captured CUDA graphs (gsis_options.capture_graphs)
    unless its request's options say otherwise.
    """

    def __init__(self, memory_budget, slots=4, precision="f32", nsm=None, make_solver=None, footprint=None,
                 new_stream=None, clock=time.perf_counter, idle=lambda s: time.sleep(min(s, 0.01)), graphs=False):
        self.memory_budget = int(memory_budget)
        self.slots = int(slots)
        self.precision = precision
        self.graphs = bool(graphs)
        if nsm is None:
            import torch
            nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        self.macro_sms = max(1, nsm // self.slots)
        self._make = make_solver or _gpu_solver
        self._footprint = footprint or _gpu_footprint
        self._new_stream = new_stream or _gpu_stream
        self._clock = clock
        self._idle = idle

    def run(self, requests):
        """Serve the requests (arrival times relative to the call) and return their results in
        request order.  A request whose footprint exceeds the whole budget is rejected (None)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        queue, running, results = [], [], {}
        used = 0
        t0 = self._clock()
        while pending or queue or running:
            now = self._clock() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.pop(0))
            while queue and len(running) < self.slots:
                req = queue[0]
                need = self._footprint(req.problem, self.precision, **req.opts)
                if need > self.memory_budget:
                    queue.pop(0)
                    results[req.rid] = None
                    continue
                if used + need > self.memory_budget:
                    break
                queue.pop(0)
                stream = self._new_stream()
                opts = dict(req.opts)
                if self.graphs:
                    opts.setdefault("capture_graphs", 1)
                solver = self._make(req.problem, self.precision, self.macro_sms, stream, **opts)
                used += need
                running.append(_Running(req, solver, stream, need, self._clock() - t0))
            if not running:
                if pending:
                    self._idle(max(0.0, pending[0].arrival - (self._clock() - t0)))
                continue
            # one round: enqueue every running solve's step, then wait for each.  A solve that fails
            # (its state left the physical range, or its steps could not be enqueued) leaves with
            # its error; the others go on.
            failed = {}
            for r in running:
                try:
                    r.solver.step_async()
                except Exception as e:  # noqa: BLE001 - the request fails, the server does not
                    failed[id(r)] = str(e)
            for r in running:
                if id(r) in failed:
                    continue
                try:
                    r.eps = r.solver.step_wait()
                except Exception as e:  # noqa: BLE001
                    failed[id(r)] = str(e)
                    continue
                r.steps += 1
                if r.eps < r.best:
                    r.best, r.since_best = r.eps, 0
                else:
                    r.since_best += 1
            done = [r for r in running if id(r) in failed or r.eps < r.req.tol or r.steps >= r.req.max_steps
                    or r.since_best >= r.req.stall_steps]
            for r in done:
                t = self._clock() - t0
                if id(r) in failed:
                    results[r.req.rid] = Result(r.req.rid, r.req.arrival, r.admitted, t, r.steps, r.eps, False,
                                                None, error=failed[id(r)])
                else:
                    conv = r.eps < r.req.tol
                    results[r.req.rid] = Result(r.req.rid, r.req.arrival, r.admitted, t, r.steps, r.eps, conv,
                                                r.solver.W(), floor=not conv and r.since_best >= r.req.stall_steps)
                r.solver.close()
                used -= r.need
                running.remove(r)
        return [results.get(r.rid) for r in sorted(requests, key=lambda r: r.rid)]


def summary(results, wall_seconds):
    """p50 / p99 latency (arrival to finished state) and solves per hour over the run, over the
    requests that finished without an error."""
    ok = [r for r in results if r is not None and not r.error]
    lat = [r.latency for r in ok]
    return {"requests": len(results), "served": len(ok), "converged": sum(r.converged for r in ok),
            "at_precision_floor": sum(r.floor for r in ok),
            "failed": sum(1 for r in results if r is not None and r.error),
            "p50_latency_s": percentile(lat, 50), "p99_latency_s": percentile(lat, 99),
            "solves_per_hour": 3600.0 * len(ok) / wall_seconds if wall_seconds > 0 else float("nan"),
            "wall_s": wall_seconds}


def _gpu_solver(problem, precision, macro_sms, stream, **opts):
    import torch

    from . import gsis

    opts = dict(opts)
    mode = opts.pop("mode", "gsis")
    with torch.cuda.stream(stream):
        return gsis.Solver(problem, precision=precision, mode=mode, macro_sms=macro_sms, **opts)


def _gpu_footprint(problem, precision, **opts):
    from . import gsis

    opts = dict(opts)
    mode = opts.pop("mode", "gsis")
    return gsis.footprint_bytes(problem, precision, mode=gsis.MODE_GSIS if mode == "gsis" else gsis.MODE_DVM, **opts)


def _gpu_stream():
    import torch

    return torch.cuda.Stream()


def poisson_requests(n, mean_gap, seed, make_problem, tol=1e-6, max_steps=400, stall_steps=20):
    """n requests with exponential inter-arrival times of mean mean_gap (seeded); make_problem(rng)
    draws each request's problem, or a (problem, solver options) pair."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for i in range(n):
        t += rng.exponential(mean_gap)
        drawn = make_problem(rng)
        prob, opts = drawn if isinstance(drawn, tuple) else (drawn, {})
        out.append(Request(i, prob, t, tol, max_steps, stall_steps, dict(opts)))
    return out

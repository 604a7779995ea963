"""Benchmark: phase-space updates per second of the GSIS solver on the 2D lid-driven cavity
(128 x 128 cells, 32^3 velocities on [-5, 5]^3 = 537M phase-space points, Kn = 0.1, lid 0.16).

The headline is the plain FP64 path (FP64 VDF, FP64 kinetic arithmetic, FP64 synthetic solve).
The same line carries the FP32- and BF16-storage forms beside it (FP32 kinetic arithmetic with
compensated FP32 moments, FP64 synthetic solve): their updates/s, their time to eps < 1e-6 (or
to their storage round-off floor) and the relative L2 distance of their converged density and
temperature from the FP64 solution.

One step = one outer GSIS iteration (Algorithm 1): wall pre-pass, fused kinetic step,
moments, FP64 synthetic solve (300 inner steps), residual and the next state.  The VDF (4.3 GB
in FP64) is far larger than L2 (129 MB), so no L2 flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica on its own GPU ("replicas only").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CFG = dict(n=128, nv=32, vmax=5.0, Kn=0.1, lid=0.16, model="shakhov")
CFG_DEFAULT_KN = CFG["Kn"]
METRIC = "phase-space updates/s (GSIS outer step, 2D cavity)"
UNIT = "updates/s"

# FP64 arithmetic of one inner step of the synthetic solve per cell, 2D monatomic (five
# conserved fields, four faces per cell), counted from the scheme's formulas (+ - * / sqrt exp
# log as one flop each): gradients and limiters 490, face fluxes 350, four red/black sweeps with
# the residual, update and axis-flux increments 716.
MACRO_FLOPS_PER_CELL_STEP_2D = 1556
# Arithmetic of the kinetic step per phase-space point, 2D Shakhov, counted from the formulas
# in the same way (comparisons, min / max and selections not counted): the correction of
# Eq. updatef on load (two Maxwellians and the combination) 25, the LSQ gradient of two axes 10,
# the Venkatakrishnan limiter 34, the Shakhov reference distribution 11 beyond the Maxwellian it
# shares with the correction, the collision and flux terms of the delta form 19, the division by
# the implicit diagonal, the update and the published face increments 4.
KINETIC_FLOPS_PER_POINT_2D = 103
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the 128^2 cavity with
# 32^3 velocities, keyed by kernel, precision and the SHA-256 prefix of the kernel's source file
# at capture time: a figure whose source has changed since is reported as null (stale).  Captured
# on the 64^2 case in the same launch configuration as at 128^2 (FP64: the colour ring in device
# scratch; FP32 and BF16: in shared memory) and scaled by the 4x cells: the kinetic kernel's
# traffic is per point, the synthetic solve's per cell (profiles/dram_bytes_cavity64x32.md).
DRAM_BYTES_PER_LAUNCH = {
    ("kinetic_kernel", "f64"): (4 * (1.0845e9 + 1.1232e9), "03162e244003"),
    ("kinetic_kernel", "f32"): (4 * (0.5405e9 + 0.4760e9), "03162e244003"),
    ("kinetic_kernel", "bf16"): (4 * (0.2706e9 + 0.2124e9), "03162e244003"),
    ("macro_kernel", "f64"): (4 * (3.79e6 + 0.02e6), "02e3bb610d02"),
}
KERNEL_SOURCES = {"kinetic_kernel": "kinetic.cu", "moments_kernel": "kinetic.cu", "macro_kernel": "macro.cu"}


def source_sha(kernel):
    path = os.path.join(ROOT, "paper_2310_18916_gb300", "csrc", KERNEL_SOURCES[kernel])
    with open(path, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:12]


def traffic(kernel, precision):
    """Measured DRAM bytes per launch, or None when not captured for this source."""
    rec = DRAM_BYTES_PER_LAUNCH.get((kernel, precision))
    if rec is None or rec[1] != source_sha(kernel):
        return None
    return rec[0]


def workload_name(c=CFG):
    gas = "" if c["model"] == "shakhov" else ", Rykov N2-like gas (two reduced VDFs)"
    return (f"2D lid-driven cavity {c['n']}x{c['n']} cells, {c['nv']}^3 velocities on [-{c['vmax']},{c['vmax']}]^3, "
            f"Kn={c['Kn']}, lid {c['lid']}{gas}")


def problem(c=CFG):
    from paper_2310_18916_gb300 import workloads as wl
    p = wl.cavity(n=c["n"], nv=c["nv"], vmax=c["vmax"], Kn=c["Kn"], lid=c["lid"])
    return wl.as_rykov(p) if c["model"] == "rykov" else p


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples (the JSON line carries their summary); CLOCKS_DIR keeps them elsewhere
        self.path = os.path.join(os.environ.get("CLOCKS_DIR", tempfile.gettempdir()), f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured", float(d.get("sm_max_mhz", 2070.0))
    return 6800.0, "fallback", 2070.0


def fp64_peak_tflops():
    """Measured FP64 rate of this GPU: cuBLAS DGEMM (torch.matmul on float64), 6144^3, best of
    three after a warm-up, CUDA events (2 n^3 flops per product)."""
    import torch

    n = 6144
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = a @ b
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        c = a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b, c
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / best / 1e12


def oracle_outer_steps(p, steps, threads):
    """Complete FP64 oracle outer steps (kinetic step over every point, moments, the 300 inner
    synthetic steps, residual and correction) of problem p, each timed; creation untimed."""
    from oracle.oracle import Oracle

    o = Oracle(p, mode=0, nthreads=threads)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        o.step()
        times.append(time.perf_counter() - t0)
    return times


SAMPLE_CELLS = 16  # the bounded CPU sample: a 16 x 16 cavity with the workload's velocity grid


def sample_problem(c=CFG):
    """The workload's cavity at 16 x 16 cells with the same velocity grid, lid, Kn and gas: the
    same 32768 velocities per cell, so the kinetic work per point and the synthetic solve's work
    per point (cells / points) are those of the full workload."""
    return problem(dict(c, n=SAMPLE_CELLS))


def cpu_baseline(c=CFG):
    """The oracle as it stands on the host cores: one complete outer step of the full workload
    on every core, and two complete outer steps of the 16 x 16 sample on one thread."""
    cores = os.cpu_count() or 1
    p = problem(c)
    nvdf = 2 if c["model"] == "rykov" else 1
    full = oracle_outer_steps(p, 1, cores)[0]
    q = sample_problem(c)
    one = oracle_outer_steps(q, 2, 1)
    qpts = q.ncells * q.nvel * nvdf
    return {"value": p.ncells * p.nvel * nvdf / full, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one complete FP64 outer step (300 inner synthetic steps) of the full {c['n']}^2 x {c['nv']}^3 "
                      f"workload on {cores} threads, timed: {full:.1f} s (creation untimed)",
            "single_thread": {"value": qpts * len(one) / sum(one), "unit": UNIT, "cores": 1, "kind": "oracle",
                              "sample": f"two complete FP64 outer steps of the {SAMPLE_CELLS}x{SAMPLE_CELLS}-cell cavity "
                                        f"with the same {c['nv']}^3 velocities ({qpts} points), timed: "
                                        f"{sum(one):.1f} s"}}


def time_to_steady(p, prec, tol, max_steps, stall=20):
    """Wall time from solver creation (host inputs) to eps < tol for one VDF precision, on one GPU.
    Stops at the first of eps < tol, a stall of eps (its storage round-off floor: `stall` steps
    without a new minimum) or max_steps.  Returns the record and the final state W."""
    import torch

    from paper_2310_18916_gb300 import gsis

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = gsis.Solver(p, precision=prec, mode="gsis")
    best, since, hist = float("inf"), 0, []
    for _ in range(max_steps):
        e = s.step()
        hist.append(e)
        if e < best:
            best, since = e, 0
        else:
            since += 1
        if e < tol or since >= stall:
            break
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    W = s.W()
    s.close()
    del s
    torch.cuda.empty_cache()
    return {"precision": prec, "tol": tol, "reached": hist[-1] < tol, "steps": len(hist), "seconds": sec,
            "eps_last": hist[-1], "eps_min": min(hist)}, W


def against_fp64(W, ref, vol):
    """Relative L2 (volume-weighted) of density and temperature and the largest velocity
    difference over the largest speed, against the FP64 solution."""
    import numpy as np

    rl2 = lambda a, b: float(np.sqrt(((a - b) ** 2 * vol).sum() / (b ** 2 * vol).sum()))
    return {"rho": rl2(W[:, 0], ref[:, 0]), "T": rl2(W[:, 4], ref[:, 4]),
            "u_max_abs_over_max": float(np.abs(W[:, 1:3] - ref[:, 1:3]).max() / np.abs(ref[:, 1:3]).max())}


def run_time_to_steady(args):
    """Time to eps < tol per VDF precision (FP64, FP32, BF16) with the accuracy of the FP32 / BF16
    solutions against the plain FP64 one."""
    import numpy as np
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    p = problem()
    vol = np.full(p.ncells, 1.0 / p.ncells)
    out, ref = [], None
    for prec in ("f64", "f32", "bf16"):
        rec, W = time_to_steady(p, prec, args.tts_tol, args.tts_max_steps)
        if prec == "f64":
            ref = W
        else:
            rec["rel_l2_vs_f64"] = against_fp64(W, ref, vol)
        out.append(rec)
    print(json.dumps({"metric": "time to steady state (GSIS, 2D cavity, from host inputs)", "unit": "s",
                      "higher_is_better": False, "config": {"workload": workload_name()}, "results": out}))
    return 0


def run_couette(args):
    """Planar Couette flow (100 cells, 24^3 velocities on [-5, 5]^3, Shakhov, omega 0.81, Kn 0.1,
    plates at -/+0.2, diffuse at T0), FP64 GSIS to eps < 1e-8: the GPU path from host inputs and
    the FP64 oracle on the host cores (the timed CPU baseline of this configuration), their step
    counts, and the agreement of the states step by step over the first steps."""
    import numpy as np
    import torch

    from oracle.oracle import Oracle
    from paper_2310_18916_gb300 import gsis
    from paper_2310_18916_gb300 import workloads as wl

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    p = wl.couette(n_cells=100, nv=24, Kn=args.kn if args.kn != CFG_DEFAULT_KN else 0.1)
    tol, max_steps, parity_steps = 1e-8, 400, 5
    cores = os.cpu_count() or 1
    # step-by-step agreement (same presteps and options on both sides)
    g = gsis.Solver(p, precision="f64", mode="gsis")
    o = Oracle(p, mode=0, nthreads=cores)
    o.presteps(10)
    worst = 0.0
    for _ in range(parity_steps):
        g.step()
        o.step()
        Wg, Wo = g.W(), o.W()
        scale = np.maximum(np.abs(Wo).max(axis=0), 1e-12)
        worst = max(worst, float((np.abs(Wg - Wo) / scale)[:, [0, 2, 4]].max()))
    g.close()
    del g, o
    torch.cuda.synchronize()
    # GPU FP64 from host inputs to eps < tol
    t0 = time.perf_counter()
    g = gsis.Solver(p, precision="f64", mode="gsis")
    done, eps_g, _ = g.iterate(max_steps, tol)
    torch.cuda.synchronize()
    gpu_s = time.perf_counter() - t0
    Wg = g.W()
    g.close()
    # oracle on the host cores, bounded to about two minutes
    t0 = time.perf_counter()
    o = Oracle(p, mode=0, nthreads=cores)
    o.presteps(10)
    hist = []
    while len(hist) < max_steps and (not hist or hist[-1] >= tol) and time.perf_counter() - t0 < 120.0:
        hist.append(o.step())
    orc_s = time.perf_counter() - t0
    Wo = o.W()
    reached = bool(hist) and hist[-1] < tol
    res = {"metric": "Couette flow to eps < 1e-8, FP64 (GPU vs oracle on the host cores)", "unit": "s",
           "higher_is_better": False,
           "config": {"workload": f"planar Couette flow, 100 cells, 24^3 velocities on [-5,5]^3, Shakhov, "
                                  f"omega 0.81, Kn {p.Kn}, plates -/+0.2", "tol": tol},
           "gpu_f64": {"seconds": gpu_s, "steps": done, "eps_last": eps_g},
           "oracle_f64": {"seconds": orc_s, "steps": len(hist), "eps_last": hist[-1] if hist else None,
                          "reached": reached, "cores": cores, "kind": "oracle"},
           "per_step_max_rel_diff_first_steps": {"steps": parity_steps, "rho_uy_T": worst},
           "final_max_rel_diff_rho_uy_T": float((np.abs(Wg - Wo) / np.maximum(np.abs(Wo).max(axis=0), 1e-12))
                                                [:, [0, 2, 4]].max()) if reached else None}
    if reached:
        res["speedup_gpu_over_oracle"] = orc_s / gpu_s
    print(json.dumps(res))
    return 0


# Bodies on general (curvilinear) O-grids: the kinetic iteration (DVM mode) with two colour
# passes per step and a pseudo-time step (1/dt = 1000: an impulsive Ma-4 start on the sphere
# keeps a positive density in the wake for the steps timed here), FP32 / BF16 storage.
BODIES = {
    # sphere of diameter 1: 32 radial (first 0.0224, ratio 1.1, R_out 5) x 24 polar x 48 azimuthal
    # cells, Ma 4, Kn 0.05, 48^3 velocities on [-12, 12]^3 clustered about the free stream
    "sphere": dict(kind="sphere", n=(32, 24, 48), nv=48, vmax=12.0, Ma=4.0, Kn=0.05, first=0.0224, R_out=5.0,
                   clustered=True),
    # the same sphere on a locally refined unstructured velocity set (truncation sphere about the
    # post-shock velocity, refined about the free stream and the wall velocity)
    "sphere_vset": dict(kind="sphere", n=(32, 24, 48), nv=4, vmax=12.0, Ma=4.0, Kn=0.05, first=0.0224, R_out=5.0,
                        vset=dict(n_base=16, refine=3)),
    # cylinder of diameter 1 in cross flow: 64 radial (first 0.01, R_out 10) x 128 azimuthal cells,
    # Ma 2, Kn 0.05, 40^3 velocities on [-9, 9]^3
    "cylinder": dict(kind="cylinder", n=(64, 1, 128), nv=40, vmax=9.0, Ma=2.0, Kn=0.05, first=0.01, R_out=10.0),
    # subsonic cylinder for the GSIS outer step on a body (Euler presteps, then GSIS): 64 x 128
    # cells, Ma 0.5, Kn 0.05, 40^3 velocities on [-6, 6]^3
    "cylinder_gsis": dict(kind="cylinder", n=(64, 1, 128), nv=40, vmax=6.0, Ma=0.5, Kn=0.05, first=0.01, R_out=10.0,
                          mode="gsis", euler_presteps=300),
    # capsule forebody (heat-shield cap of radius 1, 33 deg conical afterbody): 50 radial x 40 polar
    # x 50 azimuthal cells (100,000), diatomic Rykov gas (two reduced VDFs), Ma 10, Kn 0.01, wall at
    # 0.3 T0, 48^3 velocities clustered about the free stream on [-16, 16]^3 (1.1e10 points)
    "capsule": dict(kind="capsule", n=(50, 40, 50), nv=48, vmax=None, Ma=10.0, Kn=0.01, first=None, R_out=6.0,
                    T_w=0.3, oracle_nv=8),
    # the capsule at 1/8 of the cells with 24^3 velocities, the size its oracle parity runs at
    "capsule_small": dict(kind="capsule", n=(25, 20, 25), nv=24, vmax=None, Ma=10.0, Kn=0.01, first=None,
                          R_out=6.0, T_w=0.3, oracle_nv=8),
    # configuration 3 in GSIS: the same sphere and velocity box, reached by Mach continuation
    # 0.5 -> 1 -> ... -> 4 in steps of 0.5 (each stage from the previous converged state; the first
    # from 300 Euler presteps) with positive face values, every stage to eps < 1e-6
    "sphere_gsis": dict(kind="sphere", n=(32, 24, 48), nv=48, vmax=12.0, Ma=4.0, Kn=0.05, first=0.0224, R_out=5.0,
                        clustered=True, mode="continuation", stages=(0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0),
                        euler_presteps=300),
    # GSIS on an unstructured mesh with simplices: the lid-driven cavity of 64 x 64 squares, the
    # half with x < 1/2 split into two triangles each, extruded one layer (prisms and hexahedra,
    # 6144 cells), 32^3 velocities, Kn 0.1, two colour passes in each octant's upwind order
    "hybrid_cavity": dict(kind="hybrid", n=64, nv=32, vmax=5.0, lid=0.16, Kn=0.1, hybrid=0.5, mode="gsis",
                          euler_presteps=0, n_sweeps=2),
    # configuration 4 in GSIS: the capsule and its cold Rykov wall reached by Mach continuation
    # 1 -> 2 -> 2.5 -> ... -> 5 -> 6 -> ... -> 10 (the velocity box of each stage from its own Mach
    # number; 2 -> 3 in one stage diverges), positive face values, each stage to eps < 1e-6 or until
    # eps stops falling; reference area pi (radius 1).  Converges at Ma 1 and 2; fails above 2.5.
    "capsule_gsis": dict(kind="capsule", n=(50, 40, 50), nv=48, vmax=None, Ma=10.0, Kn=0.01, first=None, R_out=6.0,
                         T_w=0.3, mode="continuation",
                         stages=(1.0, 2.0, 2.5, 3.0, 3.5, 4.0, 4.5, 5.0, 6.0, 7.0, 8.0, 9.0, 10.0),
                         euler_presteps=300, ref_area=3.141592653589793),
    # the same with the state update relaxed by 0.5 (R36) up to Ma 4: converges to Ma 3, fails at 3.5
    "capsule_gsis_relaxed": dict(kind="capsule", n=(50, 40, 50), nv=48, vmax=None, Ma=4.0, Kn=0.01, first=None,
                                 R_out=6.0, T_w=0.3, mode="continuation", stages=(1.0, 2.0, 2.5, 3.0, 3.5, 4.0),
                                 euler_presteps=300, ref_area=3.141592653589793, relax=0.5),
    # the sphere at profiling size: 16 x 12 x 24 cells, 32^3 velocities (151M points)
    "sphere_small": dict(kind="sphere", n=(16, 12, 24), nv=32, vmax=12.0, Ma=4.0, Kn=0.05, first=0.05, R_out=5.0),
}
BODY_SWEEPS, BODY_INV_DT = 2, 1000.0


def body_problem(name, Ma=None):
    from paper_2310_18916_gb300 import workloads as wl

    b = dict(BODIES[name])
    if Ma is not None:
        b["Ma"] = Ma
    if b["kind"] == "capsule":
        return wl.capsule(n_r=b["n"][0], n_pol=b["n"][1], n_az=b["n"][2], nv=b["nv"], R_out=b["R_out"],
                          first=b["first"], Ma=b["Ma"], Kn=b["Kn"], T_w=b["T_w"], vmax=b["vmax"])
    if b["kind"] == "hybrid":
        return wl.unstructured_cavity(n=b["n"], nv=b["nv"], vmax=b["vmax"], lid=b["lid"], Kn=b["Kn"],
                                      hybrid=b["hybrid"])
    if b["kind"] == "sphere":
        p = wl.sphere(n_r=b["n"][0], n_pol=b["n"][1], n_az=b["n"][2], nv=b["nv"], R=0.5, R_out=b["R_out"],
                      first=b["first"], Ma=b["Ma"], Kn=b["Kn"], vmax=b["vmax"])
        if b.get("clustered"):
            p = wl.with_clustered_velocities(p, b["nv"], b["vmax"])
        if b.get("vset"):
            p = wl.with_velocity_set(p, wl.hybrid_velocity_set(p.wall_u[1], T_inf=1.0, T_w=p.wall_T[0], **b["vset"]))
        return p
    return wl.cylinder(n_r=b["n"][0], n_theta=b["n"][2], nv=b["nv"], R=0.5, R_out=b["R_out"], first=b["first"],
                       Ma=b["Ma"], Kn=b["Kn"], vmax=b["vmax"])


def run_body(args):
    """Kinetic iteration on a body-fitted O-grid (the general-mesh path): phase-space updates/s,
    the general kinetic kernel's HBM roofline, the end-to-end figure through the public API and
    the oracle's CPU baseline on a bounded sample (fewer velocities)."""
    import numpy as np
    import torch

    from paper_2310_18916_gb300 import gsis
    from paper_2310_18916_gb300 import workloads as wl

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    p = body_problem(args.body)
    nvdf = 2 if p.model == wl.RYKOV else 1   # a phase-space update counts each reduced VDF's point
    pts = p.ncells * p.nvel * nvdf
    b = BODIES[args.body]
    mode = b.get("mode", "dvm")
    if mode == "gsis":
        kw = dict(precision=args.precision, mode="gsis", n_sweeps=b.get("n_sweeps", BODY_SWEEPS),
                  euler_presteps=b["euler_presteps"])
    else:
        kw = dict(precision=args.precision, mode="dvm", n_sweeps=BODY_SWEEPS, kin_inv_dt=BODY_INV_DT)
    if args.graphs:
        kw["capture_graphs"] = 1
    s = gsis.Solver(p, kinetic_presteps=0, **kw)
    for _ in range(args.warmup):
        s.step()
    if not args.graphs:
        s.profile(True, reset=True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            s.step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms_total = e0.elapsed_time(e1)
    if args.graphs:
        # graph replays carry no phase events: the phase split of two more steps, launched directly
        graphs_held = s.graphs()
        s.profile(True, reset=True)
        for _ in range(2):
            s.step()
    phase, nsteps, launches = s.profile(False)
    eps = float(s.residual()[3])
    W = s.W()
    s.close()
    del s
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    s2 = gsis.Solver(p, kinetic_presteps=0, **kw)
    for _ in range(args.steps):
        s2.step()
        W2 = s2.W()
    s2.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    del s2
    peak, peak_kind, _ = measured_peaks()
    sbytes = {"f32": 4, "f64": 8, "bf16": 2}[args.precision]
    kin_ms = phase[1] / max(nsteps, 1)
    ms = ms_total / args.steps
    line = {
        "metric": f"phase-space updates/s ({'GSIS outer step' if mode == 'gsis' else 'kinetic iteration'}, "
                  f"{b['kind']} {'mesh' if p.ucells is not None else 'O-grid'})",
        "value": pts * args.steps / (ms_total / 1e3),
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "f64" else "f32", "data": "synthetic",
        "config": {"workload": f"{p.name}: {BODIES[args.body]}", "precision": f"{args.precision} VDF",
                   "cuda_graphs": (graphs_held if args.graphs else False),
                   "cells": p.ncells, "velocities": p.nvel, "vdfs": nvdf, "points": pts, "n_sweeps": kw["n_sweeps"],
                   "mode": mode, "kin_inv_dt": kw.get("kin_inv_dt", 0.0),
                   "euler_presteps": kw.get("euler_presteps", 0), "parallelism": "1 GPU",
                   "l2": f"inputs larger than L2 (VDF {pts * sbytes / 1e9:.2f} GB)", "eps_last": eps,
                   "rho_range": [float(W[:, 0].min()), float(W[:, 0].max())]},
        "phase_ms_per_step": {k: v / max(nsteps, 1) for k, v in zip(
            ("wall_prepass", "kinetic", "reduce_moments", "synthetic_fp64", "residual_state"), phase)},
        "roofline": {"kernel": "kinetic_general_kernel", "bound": "hbm",
                     "achieved": 2 * sbytes * pts / (kin_ms / 1e3) / 1e9, "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": 2 * sbytes * pts / (kin_ms / 1e3) / 1e9 / peak,
                     "traffic": None, "algorithmic_bytes_per_launch": 2 * sbytes * pts, "launch_ms": kin_ms,
                     "share_of_step": kin_ms / ms},
        "e2e": {"value": pts * args.steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": ((p.unodes.nbytes + p.ucells.nbytes if p.ucells is not None else p.nodes.nbytes)
                                       + 6 * p.vx.nbytes + (p.W0.nbytes if p.W0 is not None else 0)) / args.steps,
                "d2h_bytes_per_step": W2.nbytes, "seconds": e2e_s,
                "includes": "create from host inputs, steps, per-step state read, destroy"},
        "gpu_launches": launches / max(nsteps, 1) * args.steps,
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = body_oracle_sample(args.body)
    print(json.dumps(line))
    return 0


def run_body_continuation(args):
    """GSIS on a body-fitted grid from the free stream at the target Mach number, reached by Mach
    continuation: each stage starts from the previous stage's converged state (its Maxwellian,
    then 10 kinetic presteps) with a faster free stream, and runs GSIS outer steps (two colour
    passes, positive face values, the configured update relaxation) to eps < 1e-6, or until eps
    stops falling for 15 steps.
    Reports the time to the converged target state (creation and presteps included), the GSIS
    outer-step throughput of the last stage (CUDA events), its phase split and the drag and
    heat-flux coefficients."""
    import numpy as np
    import torch

    from paper_2310_18916_gb300 import gsis
    from paper_2310_18916_gb300 import workloads as wl

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    b = BODIES[args.body]
    W, stages, t_all = None, [], 0.0
    with ClockSampler(local) as clk:
        for Ma in b["stages"]:
            p = body_problem(args.body, Ma=Ma)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            euler = b.get("euler_presteps", 0) if W is None else 0
            try:
                s = gsis.Solver(p, precision=args.precision, mode="gsis", n_sweeps=BODY_SWEEPS, init_W=W,
                                positive_faces=1, euler_presteps=euler, relax=b.get("relax", 0.0),
                                kinetic_presteps=10 if W is None else b.get("stage_presteps", 10))
            except gsis.GsisError as err:
                stages.append({"Ma": Ma, "error": str(err)})
                break
            s.profile(True, reset=True)
            stream = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            best, since, hist, failed = np.inf, 0, [], None
            for _ in range(args.steps if args.steps > 20 else 80):
                try:
                    e = s.step()
                except gsis.GsisError as err:
                    failed = str(err)
                    break
                hist.append(e)
                best, since = (e, 0) if e < best else (best, since + 1)
                if e < 1e-6 or since >= 15:
                    break
            e1.record(stream)
            torch.cuda.synchronize()
            if failed or not hist:
                s.close()
                stages.append({"Ma": Ma, "steps": len(hist), "error": failed or "no step",
                               "eps_history": [float(h) for h in hist]})
                break
            wall = time.perf_counter() - t0
            phase, nsteps, launches = s.profile(False)
            U = float(np.linalg.norm(p.wall_u[1]))
            loads = s.wall_loads([0], (1.0, 0.0, 0.0), 1.0, U, b.get("ref_area", np.pi * 0.5 ** 2))
            W = s.W()
            s.close()
            t_all += wall
            stages.append({"Ma": Ma, "steps": len(hist), "eps_last": hist[-1], "reached": hist[-1] < 1e-6,
                           "seconds": wall, "ms_per_step_device": e0.elapsed_time(e1) / len(hist),
                           "phase_ms_per_step": {k: v / max(nsteps, 1) for k, v in zip(PHASES, phase)},
                           "C_D": float(loads[4]), "C_H": float(loads[5]), "rho_min": float(W[:, 0].min())})
    if "error" in stages[-1]:
        print(json.dumps({"metric": f"phase-space updates/s (GSIS outer step, {b['kind']} O-grid, Mach continuation)",
                          "value": None, "unit": UNIT, "failed_stage": stages[-1], "stages": stages,
                          "config": {"workload": f"{p.name}: {b}", "precision": args.precision}}))
        return 1
    last = stages[-1]
    pts = p.ncells * p.nvel * (2 if p.model == wl.RYKOV else 1)   # both reduced VDFs for Rykov
    peak, peak_kind, _ = measured_peaks()
    sbytes = {"f32": 4, "f64": 8, "bf16": 2}[args.precision]
    kin_ms = last["phase_ms_per_step"]["kinetic"]
    line = {
        "metric": f"phase-space updates/s (GSIS outer step, {b['kind']} O-grid, Mach continuation)",
        "value": pts / (last["ms_per_step_device"] / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": last["steps"], "warmup": 0, "ms_per_step": last["ms_per_step_device"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "f64" else "f32",
        "data": "synthetic",
        "config": {"workload": f"{p.name}: {b}", "precision": f"{args.precision} VDF, f64 synthetic solve",
                   "cells": p.ncells, "velocities": p.nvel, "points": pts, "n_sweeps": BODY_SWEEPS,
                   "positive_faces": 1, "stages": list(b["stages"]), "parallelism": "1 GPU",
                   "l2": f"inputs larger than L2 (VDF {pts * sbytes / 1e9:.2f} GB)"},
        "time_to_steady_s": t_all, "stages": stages,
        "roofline": {"kernel": "kinetic_general_kernel", "bound": "hbm",
                     "achieved": 2 * sbytes * pts / (kin_ms / 1e3) / 1e9, "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": 2 * sbytes * pts / (kin_ms / 1e3) / 1e9 / peak, "traffic": None,
                     "algorithmic_bytes_per_launch": 2 * sbytes * pts, "launch_ms": kin_ms},
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    return 0


def body_oracle_sample(name):
    """The oracle on the same mesh with 12^3 velocities (8^3 on the capsule; one step of the same
    mode, all host cores; the Euler presteps of a GSIS body untimed), scaled to updates/s."""
    import numpy as np

    from oracle.oracle import Oracle
    from paper_2310_18916_gb300 import workloads as wl

    p = body_problem(name)
    b = BODIES[name]
    nvo = b.get("oracle_nv", 12)
    vmax = b["vmax"] or float(max(np.abs(p.vx).max(), np.abs(p.vy).max(), np.abs(p.vz).max()))
    v, w = wl.midpoint_grid(nvo, -vmax, vmax)
    p.vx, p.vy, p.vz, p.wx, p.wy, p.wz = v, v.copy(), v.copy(), w, w.copy(), w.copy()
    p.vpoints = None
    cores = os.cpu_count() or 1
    if b.get("mode", "dvm") == "gsis":
        o = Oracle(p, mode=0, n_sweeps=b.get("n_sweeps", BODY_SWEEPS), nthreads=cores)
        if b["euler_presteps"]:
            o.euler_presteps(b["euler_presteps"])
        what = "GSIS outer step (300 inner synthetic steps at most)"
    else:
        o = Oracle(p, mode=1, n_sweeps=BODY_SWEEPS, kin_inv_dt=BODY_INV_DT, nthreads=cores)
        what = "kinetic-iteration step"
    t0 = time.perf_counter()
    o.step()
    dt = time.perf_counter() - t0
    nvdf = 2 if p.model == wl.RYKOV else 1
    return {"value": p.ncells * p.nvel * nvdf / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one {what} of the same mesh with {nvo}^3 velocities ({dt:.1f} s)"}


def run_serve(args):
    """Configuration 5 scaled to minutes: a seeded Poisson stream of steady solves, cavities and
    cylinders with equal odds (sizes, velocity counts and arrival gaps scaled down; Kn
    log-uniform in [1e-3, 1]; lid Mach number in [0.1, 5], cylinders subsonic; GSIS below Kn 0.3,
    the plain kinetic iteration above), served with continuous batching in FP32, against the same
    requests solved one at a time in FP32 and in plain FP64."""
    import torch

    from paper_2310_18916_gb300 import serving
    from paper_2310_18916_gb300 import workloads as wl

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    reqs = serving.poisson_requests(args.serve_requests, args.serve_gap, 0,
                                    lambda rng: wl.serving_request(rng, sizes=(32, 48, 64), nvs=(16, 20, 24)),
                                    tol=1e-6, max_steps=150)
    budget = int(0.5 * torch.cuda.mem_get_info()[0])
    lines = {}
    for name, slots, prec, arrivals, graphs in (("batched_f32", args.serve_slots, "f32", True, False),
                                                ("sequential_f32", 1, "f32", False, False),
                                                ("sequential_f64", 1, "f64", False, False)):
        rs = reqs if arrivals else [serving.Request(r.rid, r.problem, 0.0, r.tol, r.max_steps, r.stall_steps, r.opts)
                                    for r in reqs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = serving.Server(budget, slots=slots, precision=prec, graphs=graphs).run(rs)
        wall = time.perf_counter() - t0
        summ = serving.summary(res, wall)
        summ["slots"] = slots
        summ["precision"] = prec
        summ["cuda_graphs"] = graphs
        summ["failures"] = [{"rid": r.rid, "problem": reqs[r.rid].problem.name, "opts": reqs[r.rid].opts,
                             "error": r.error} for r in res if r is not None and r.error]
        lines[name] = summ
    b = lines["batched_f32"]
    kinds = {"cavity": sum(r.problem.name.startswith("cavity") for r in reqs),
             "cylinder": sum(r.problem.name.startswith("cylinder") for r in reqs),
             "gsis": sum(r.opts.get("mode") == "gsis" for r in reqs),
             "dvm": sum(r.opts.get("mode") == "dvm" for r in reqs)}
    print(json.dumps({"metric": "steady-solve serving (cavity and cylinder stream)", "unit": "s",
                      "p50_latency_s": b["p50_latency_s"], "p99_latency_s": b["p99_latency_s"],
                      "solves_per_hour": b["solves_per_hour"], "higher_is_better": False,
                      "config": {"requests": len(reqs), "mix": kinds, "mean_gap_s": args.serve_gap,
                                 "slots": args.serve_slots,
                                 "sizes": "cavities 32^2, 48^2, 64^2 cells; cylinders n x 2n, n = 32, 48, 64; "
                                          "16^3, 20^3, 24^3 velocities",
                                 "kn": "log-uniform [1e-3, 1]", "mach": "cavity lid [0.1, 5], cylinder [0.1, 1]",
                                 "mode": "GSIS below Kn 0.3, plain kinetic iteration above", "tol": 1e-6,
                                 "memory_budget_bytes": budget},
                      "runs": lines,
                      "throughput_vs_sequential_f64": b["solves_per_hour"] / lines["sequential_f64"]["solves_per_hour"],
                      "throughput_vs_sequential_f32": b["solves_per_hour"] / lines["sequential_f32"]["solves_per_hour"]}))
    return 0


def run_moments_gemm(args):
    """Could tensor cores take the moment projection?  The 16 raw velocity moments (1, xi, xi xi,
    |xi|^2 xi / 2, |xi|^2 / 2; weights folded in) of a VDF on the benchmark workload, taken as one
    GEMM F [cells x velocities] @ B [velocities x 16] by cuBLAS: FP64 (DGEMM), FP32 (SGEMM), TF32
    and BF16 tensor cores (FP32 accumulation), each on the VDF stored in that precision.  Against
    the library's own moments pass in FP64, FP32 and BF16 storage (the reduce_moments phase of
    timed GSIS steps: moments about the cell velocity, compensated sums).  Accuracy: T and q
    recovered from each GEMM's raw moments against the FP64 GEMM's.  The VDF is a seeded
    perturbed Maxwellian of the workload's shape, built on the device."""
    import numpy as np
    import torch

    from paper_2310_18916_gb300 import gsis

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    p = problem()
    nc, nv = p.ncells, p.nvel
    dev = "cuda"
    g = torch.Generator(device="cpu").manual_seed(7)
    rho = 1 + 0.05 * (2 * torch.rand(nc, 1, generator=g, dtype=torch.float64) - 1)
    u = 0.1 * (2 * torch.rand(nc, 3, generator=g, dtype=torch.float64) - 1)
    T = 1 + 0.05 * (2 * torch.rand(nc, 1, generator=g, dtype=torch.float64) - 1)
    X, Y, Z = np.meshgrid(p.vx, p.vy, p.vz, indexing="ij")
    flat = lambda a: torch.from_numpy(np.ascontiguousarray(a.transpose(2, 1, 0).ravel()))
    xi = torch.stack([flat(X), flat(Y), flat(Z)], 1).to(dev)
    w = flat(p.wx[:, None, None] * p.wy[None, :, None] * p.wz[None, None, :]).to(dev)
    rho, u, T = rho.to(dev), u.to(dev), T.to(dev)
    F64 = torch.empty((nc, nv), dtype=torch.float64, device=dev)
    for c0 in range(0, nc, 512):
        c1 = min(nc, c0 + 512)
        cc = xi[None, :, :] - u[c0:c1, None, :]
        F64[c0:c1] = rho[c0:c1] * (np.pi * T[c0:c1]) ** -1.5 * torch.exp(-(cc * cc).sum(-1) / T[c0:c1]) * \
            (1 + 0.05 * torch.sin(3 * cc[..., 0]) * torch.cos(2 * cc[..., 1]))
    x2 = (xi * xi).sum(1)
    cols = [w, w * xi[:, 0], w * xi[:, 1], w * xi[:, 2], w * xi[:, 0] ** 2, w * xi[:, 1] ** 2, w * xi[:, 2] ** 2,
            w * xi[:, 0] * xi[:, 1], w * xi[:, 0] * xi[:, 2], w * xi[:, 1] * xi[:, 2], 0.5 * w * x2 * xi[:, 0],
            0.5 * w * x2 * xi[:, 1], 0.5 * w * x2 * xi[:, 2], 0.5 * w * x2, 0 * w, 0 * w]
    B64 = torch.stack(cols, 1).contiguous()

    def derived(M):
        M = M.double()
        r = M[:, 0]
        uu = M[:, 1:4] / r[:, None]
        e = M[:, 13] / r - 0.5 * (uu * uu).sum(1)              # |c|^2 / 2 per unit mass
        Tm = e / 0.75
        # q = int |c|^2 c f / 2 from the raw moments about the origin
        Pxy = torch.stack([torch.stack([M[:, 4], M[:, 7], M[:, 8]], 1), torch.stack([M[:, 7], M[:, 5], M[:, 9]], 1),
                           torch.stack([M[:, 8], M[:, 9], M[:, 6]], 1)], 1)
        q = M[:, 10:13] - torch.einsum("cij,cj->ci", Pxy, uu) - M[:, 13:14] * uu + r[:, None] * (uu * uu).sum(1, keepdim=True) * uu
        return Tm, q

    def time_gemm(A, Bm, K=10):
        for _ in range(3):
            torch.matmul(A, Bm)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(K):
            out = torch.matmul(A, Bm)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K, out

    ms64, M64 = time_gemm(F64, B64)
    T_ref, q_ref = derived(M64)
    qs = (M64[:, 0] * T_ref ** 1.5).abs().max()
    F32 = F64.float()
    del F64
    torch.cuda.empty_cache()
    gemm = {"f64_dgemm": {"ms": ms64, "bytes": nc * nv * 8}}
    for name, A, Bm, tf32 in (("f32_sgemm", F32, B64.float(), False), ("tf32_tensor", F32, B64.float(), True),
                              ("bf16_tensor", None, B64.bfloat16(), False)):
        if A is None:
            A = F32.bfloat16()   # (the product is returned in BF16 too)
        torch.backends.cuda.matmul.allow_tf32 = tf32
        ms, M = time_gemm(A, Bm)
        Tm, q = derived(M)
        gemm[name] = {"ms": ms, "bytes": A.numel() * A.element_size(),
                      "T_max_rel_err": float(((Tm - T_ref).abs() / T_ref).max()),
                      "q_max_err_over_rho_T32": float((q - q_ref).abs().max() / qs)}
        del A
    torch.backends.cuda.matmul.allow_tf32 = False
    del F32
    torch.cuda.empty_cache()
    own = {}
    for prec in ("f64", "f32", "bf16"):
        s_ = gsis.Solver(p, precision=prec, mode="gsis", kinetic_presteps=0)
        s_.step()
        s_.profile(True, reset=True)
        for _ in range(3):
            s_.step()
        ph, n, _ = s_.profile(False)
        own[prec] = {"ms": ph[PHASES.index("reduce_moments")] / max(n, 1),
                     "bytes": nc * nv * {"f64": 8, "f32": 4, "bf16": 2}[prec]}
        s_.close()
    print(json.dumps({"metric": "moment projection: cuBLAS GEMM vs the library's moments pass", "unit": "ms",
                      "config": {"workload": workload_name(), "cells": nc, "velocities": nv,
                                 "moments": "16 raw moments about the origin (GEMM); 18 about the cell velocity "
                                            "(library, incl. the collision sums)"},
                      "gemm": gemm, "library": own}))
    return 0


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, on every host core.  Each step is one
    complete outer step (kinetic step, moments, 300 inner synthetic steps, residual) of the
    bounded sample of the workload: the cavity at 16 x 16 cells with the workload's 32^3 velocity
    grid, lid, Kn and gas, so that each update carries the same kinetic and synthetic work as at
    128^2.  W untimed steps, then K timed ones; value = points updated / time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    q = sample_problem()
    nvdf = 2 if CFG["model"] == "rykov" else 1
    qpts = q.ncells * q.nvel * nvdf
    times = oracle_outer_steps(q, args.warmup + args.steps, cores)[args.warmup:]
    total = sum(times)
    ms = 1e3 * total / args.steps
    value = qpts * args.steps / total
    desc = (f"each step one complete FP64 oracle outer step of the {SAMPLE_CELLS}x{SAMPLE_CELLS}-cell cavity with the "
            f"workload's {CFG['nv']}^3 velocities ({qpts} points), {cores} threads, timed; {args.warmup} untimed steps first")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(), "precision": "f64 (CPU oracle)", "parallelism": f"{cores} host threads",
                       "sample": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def timed_steps(p, prec, steps, warmup, barrier, local, shard_kw=None):
    """W untimed then K timed GSIS outer steps of a fresh solver on the device (CUDA events on
    the solver's stream, clocks sampled meanwhile), with the per-phase profile of the timed
    steps.  The solver is destroyed afterwards."""
    import torch

    from paper_2310_18916_gb300 import gsis

    s = gsis.Solver(p, precision=prec, mode="gsis", kinetic_ring=RING[0], **(shard_kw or {}))
    for _ in range(warmup):
        s.step()
    s.profile(True, reset=True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        for _ in range(steps):
            s.step()
        e1.record(stream)
        barrier()
    out = {"ms_total": e0.elapsed_time(e1)}
    out["phase"], out["nsteps"], out["launches"] = s.profile(False)
    out["eps"] = float(s.residual()[3])
    out["macro_iters"] = s.stats()[1]
    out["clocks"] = clk.summary()
    s.close()
    del s
    torch.cuda.empty_cache()
    return out


PHASES = ("wall_prepass", "kinetic", "reduce_moments", "synthetic_fp64", "residual_state")
RING = [0]   # gsis_options.kinetic_ring of the cavity runs (--kinetic-ring)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f64", choices=["f32", "f64", "bf16"],
                    help="VDF storage of the headline (kinetic arithmetic is FP64 for f64, FP32 for f32 and bf16)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP32 / BF16 sub-records and the time-to-steady comparison")
    ap.add_argument("--n", type=int, default=CFG["n"], help="cells per side (profiling cases use 64)")
    ap.add_argument("--nv", type=int, default=CFG["nv"], help="velocities per axis")
    ap.add_argument("--kn", type=float, default=CFG["Kn"])
    ap.add_argument("--model", default="shakhov", choices=["shakhov", "rykov"],
                    help="gas model (rykov: two reduced VDFs; a phase-space update counts each VDF's point)")
    ap.add_argument("--time-to-steady", action="store_true",
                    help="instead of the throughput line: wall time to eps < --tts-tol for FP64, FP32, BF16")
    ap.add_argument("--tts-tol", type=float, default=1e-6)
    ap.add_argument("--tts-max-steps", type=int, default=400)
    ap.add_argument("--serve", action="store_true", help="instead of the throughput line: the serving stream")
    ap.add_argument("--couette", action="store_true",
                    help="instead of the throughput line: Couette flow to eps < 1e-8 in FP64, GPU vs oracle")
    ap.add_argument("--kinetic-ring", type=int, default=0, choices=[0, 1],
                    help="gsis_options.kinetic_ring of the cavity runs: 1 keeps the kinetic sweep's colour ring "
                         "in device scratch at any size (the placement the 128^2 FP64 workload takes), for "
                         "profiling that placement on a smaller case")
    ap.add_argument("--moments-gemm", action="store_true",
                    help="instead of the throughput line: the moment projection as a cuBLAS GEMM against the "
                         "library's moments pass")
    ap.add_argument("--body", choices=sorted(BODIES),
                    help="instead of the cavity line: the kinetic iteration on a body-fitted O-grid")
    ap.add_argument("--graphs", action="store_true",
                    help="--body: run the timed outer steps as captured CUDA graphs (gsis_options.capture_graphs)")
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun: one solve sharded over the ranks' velocities (strong scaling) "
                         "instead of a replica per rank")
    ap.add_argument("--serve-requests", type=int, default=16)
    ap.add_argument("--serve-gap", type=float, default=0.25, help="mean arrival gap, seconds")
    ap.add_argument("--serve-slots", type=int, default=4)
    args = ap.parse_args()
    CFG.update(n=args.n, nv=args.nv, Kn=args.kn, model=args.model)
    RING[0] = args.kinetic_ring
    if args.impl == "reference":
        return run_reference(args)
    if args.time_to_steady:
        return run_time_to_steady(args)
    if args.serve:
        return run_serve(args)
    if args.couette:
        return run_couette(args)
    if args.body and BODIES[args.body].get("mode") == "continuation":
        return run_body_continuation(args)
    if args.body:
        return run_body(args)
    if args.moments_gemm:
        return run_moments_gemm(args)

    import numpy as np
    import torch

    from paper_2310_18916_gb300 import gsis

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    p = problem()
    nvdf = 2 if args.model == "rykov" else 1
    pts = p.ncells * p.nvel * nvdf
    sharded = args.shard and world > 1
    shard_kw = {}
    if sharded:
        from paper_2310_18916_gb300 import sharding
        shard_kw = dict(shard=(rank, world), allreduce=sharding.dist_allreduce())
    head = timed_steps(p, args.precision, args.steps, args.warmup, barrier, local, shard_kw)
    ms_total = head["ms_total"]
    if dist is not None:
        t = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms = ms_total / args.steps
    value = (1 if sharded else world) * pts * args.steps / (ms_total / 1e3)
    per = lambda rec, k: rec["phase"][PHASES.index(k)] / max(rec["nsteps"], 1)

    # end to end through the public API: create from host inputs, K steps each followed by a
    # device->host read of the state, destroy
    barrier()
    t0 = time.perf_counter()
    s2 = gsis.Solver(p, precision=args.precision, mode="gsis", kinetic_presteps=0, kinetic_ring=RING[0], **shard_kw)
    for _ in range(args.steps):
        s2.step()
        W = s2.W()
    s2.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    del s2
    torch.cuda.empty_cache()
    h2d = p.nodes.nbytes + 6 * p.vx.nbytes + p.W0.nbytes
    d2h = W.nbytes + 4 * 8

    # the FP32 / BF16 storage forms beside the FP64 headline: throughput, and time to steady
    # state with the accuracy of the result against the FP64 solution
    forms = None
    if world == 1 and args.precision == "f64" and not args.no_forms:
        vol = np.full(p.ncells, 1.0 / p.ncells)
        tts = {}
        for prec in ("f64", "f32", "bf16"):
            tts[prec] = time_to_steady(p, prec, args.tts_tol, args.tts_max_steps)
        forms = {"time_to_steady_f64": tts["f64"][0]}
        for prec in ("f32", "bf16"):
            r = timed_steps(p, prec, args.steps, args.warmup, barrier, local)
            sb = {"f32": 4, "bf16": 2}[prec]
            kin = per(r, "kinetic")
            peak, peak_kind, _ = measured_peaks()
            rec = {"value": pts * args.steps / (r["ms_total"] / 1e3), "unit": UNIT,
                   "ms_per_step": r["ms_total"] / args.steps, "steps": args.steps, "warmup": args.warmup,
                   "dtype": "f32", "storage": prec,
                   "phase_ms_per_step": {k: per(r, k) for k in PHASES},
                   "roofline_kinetic": {"kernel": "kinetic_kernel", "bound": "hbm",
                                        "achieved": 2 * sb * pts / (kin / 1e3) / 1e9, "peak": peak,
                                        "peak_kind": peak_kind, "unit": "GB/s",
                                        "frac": 2 * sb * pts / (kin / 1e3) / 1e9 / peak,
                                        "traffic": traffic("kinetic_kernel", prec),
                                        "algorithmic_bytes_per_launch": 2 * sb * pts, "launch_ms": kin},
                   "gpu_launches": r["launches"], "clocks": r["clocks"],
                   "time_to_steady": tts[prec][0],
                   "rel_l2_vs_f64": against_fp64(tts[prec][1], tts["f64"][1], vol),
                   "speedup_time_to_steady_vs_f64": tts["f64"][0]["seconds"] / tts[prec][0]["seconds"]}
            forms[prec] = rec

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    peak, peak_kind, sm_mhz = measured_peaks()
    sbytes = {"f32": 4, "f64": 8, "bf16": 2}[args.precision]
    kin_ms, macro_ms = per(head, "kinetic"), per(head, "synthetic_fp64")
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    fp64_derived = nsm * 2 * 2 * sm_mhz * 1e6 / 1e12
    try:
        fp64_meas = fp64_peak_tflops() if world == 1 else None
    except RuntimeError:
        fp64_meas = None
    fp64_peak = fp64_meas if fp64_meas else fp64_derived
    fp64_kind = ("measured: cuBLAS DGEMM 6144^3 (torch.matmul, float64), best of 3, in this run" if fp64_meas else
                 "derived: SMs x 2 FP64 FMA lanes x 2 flops x max SM clock")
    macro_flops = MACRO_FLOPS_PER_CELL_STEP_2D * p.ncells * head["macro_iters"] if nvdf == 1 else None
    vdf_gb = p.ncells * p.nvel * sbytes / 1e9
    if args.precision == "f64":
        # the dominant kernel of the FP64 step: the kinetic kernel, bound by the FP64 pipe
        kflops = KINETIC_FLOPS_PER_POINT_2D * pts if nvdf == 1 and p.nk == 1 else None
        roof = {"kernel": "kinetic_kernel", "bound": "alu",
                "achieved": kflops / (kin_ms / 1e3) / 1e12 if kflops else None, "peak": fp64_peak,
                "peak_kind": fp64_kind, "unit": "TFLOP/s",
                "frac": kflops / (kin_ms / 1e3) / 1e12 / fp64_peak if kflops else None,
                "traffic": traffic("kinetic_kernel", "f64"), "algorithmic_flops_per_launch": kflops,
                "flops_per_point": KINETIC_FLOPS_PER_POINT_2D, "launch_ms": kin_ms, "share_of_step": kin_ms / ms,
                "algorithmic_bytes_per_launch": 2 * sbytes * pts,
                "hbm_frac": 2 * sbytes * pts / (kin_ms / 1e3) / 1e9 / peak}
    else:
        roof = {"kernel": "kinetic_kernel", "bound": "hbm", "achieved": 2 * sbytes * pts / (kin_ms / 1e3) / 1e9,
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": 2 * sbytes * pts / (kin_ms / 1e3) / 1e9 / peak,
                "traffic": traffic("kinetic_kernel", args.precision), "algorithmic_bytes_per_launch": 2 * sbytes * pts,
                "launch_ms": kin_ms, "share_of_step": kin_ms / ms}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "f64" else "f32", "data": "synthetic",
        "config": {"workload": workload_name(),
                   "precision": f"{args.precision} VDF, {'f64' if args.precision == 'f64' else 'f32'} kinetic "
                                f"arithmetic, f64 synthetic solve",
                   "cells": p.ncells, "velocities": p.nvel, "points": pts,
                   "parallelism": f"velocity shards x{world}" if sharded else ("replicas" if world > 1 else "1 GPU"),
                   "l2": f"inputs larger than L2 (VDF {vdf_gb:.2f} GB)" if vdf_gb > 0.129 else
                         f"VDF {vdf_gb:.3f} GB fits in L2 (profiling size)", "macro_inner_steps": head["macro_iters"],
                   "eps_last": head["eps"]},
        "phase_ms_per_step": {k: per(head, k) for k in PHASES},
        "kinetic_updates_per_s": pts / (kin_ms / 1e3),
        "roofline": roof,
        "roofline_synthetic": {"kernel": "macro_kernel", "bound": "alu",
                               "achieved": macro_flops / (macro_ms / 1e3) / 1e12 if macro_flops else None,
                               "peak": fp64_peak, "peak_kind": fp64_kind, "unit": "TFLOP/s",
                               "frac": macro_flops / (macro_ms / 1e3) / 1e12 / fp64_peak if macro_flops else None,
                               "traffic": traffic("macro_kernel", "f64") if args.n == 128 and nvdf == 1 else None,
                               "algorithmic_flops_per_launch": macro_flops,
                               "flops_per_cell_inner_step": MACRO_FLOPS_PER_CELL_STEP_2D, "launch_ms": macro_ms,
                               "share_of_step": macro_ms / ms},
        "fp64_peak_tflops": {"measured": fp64_meas, "derived": fp64_derived},
        "e2e": {"value": (1 if sharded else world) * args.steps * pts / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": d2h, "seconds": e2e_s, "includes": "create from host inputs, steps, per-step state read, destroy"},
        "gpu_launches": head["launches"],
        "clocks": head["clocks"],
    }
    if forms is not None:
        line["forms"] = forms
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

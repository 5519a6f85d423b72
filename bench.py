#!/usr/bin/env python
"""Benchmark: time-to-solution at 1e-4 relative-L2 seismogram error, and the HBM roofline of
the fused stencil pass, on the batched workload (64 shots on a 1001 x 501 layered model
plus 8 layered models from 201 x 101 to 801 x 401; 8th order, free surface, 40-point PML,
Ricker 10 Hz, T = 2 s; FP32 wavefields, FP64 coefficients).

One "step" of this benchmark is one complete simulation of the whole batch to T (every
shot's seismogram), at the cheapest (method, m, dt) whose seismogram error against an FP64
reference is at most 1e-4 (searched in-run on sampled problems, see
paper_2401_16322_gb300/tts.py).  The inputs (state, workspace: several GB) are larger than
L2, and every simulation starts from a zeroed state.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Rank 0 prints one JSON line (strict JSON: a non-finite number is written as null).  The side
runs (FP64 single shot, FWI gradients, the 3D cube, the small FP64 study, the dispersion
table, every search candidate) are summarised in it; --detail-out PATH writes them in full.
--impl reference times the FP64 CPU oracle on a bounded sample of the same workload, on
every host core (independent shots in separate processes), and scales it to the same metric.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-solution at 1e-4 rel. L2 seismogram error; stencil HBM GB/s as % of peak"
UNIT = "s"
T_END = 2.0
TARGET = 1e-4
# Sampled problems for the error measurement: (model index, shot index).
PICKS = [(0, 32), (1, 0), (5, 0)]
# Problems on which the selected setting's error is checked after the timed region: one shot
# of every uneven model and eight shots spread over the 64 of the large model.
CHECK_PROBLEMS = [(q, 0) for q in range(1, 9)] + [(0, k) for k in (0, 9, 18, 27, 32, 36, 45, 54, 63)]
# Cheapest candidate found by the in-run search on GB300 (used by the CPU reference arm; the
# GPU arm re-runs the search and reports what it finds).
DEFAULT_SELECTION = ("hork-horner", 20, 4)     # method, m, dt in units of the leap-frog step
WORKLOAD_NAME = ("batched: 64 shots on 1001x501 + 8 models 201x101..801x401, layered "
                 "1500-4500 m/s, 8th order, free surface, 40-pt PML, Ricker 10 Hz, T=2 s")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--target", type=float, default=TARGET)
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    ap.add_argument("--no-search", action="store_true", help="use the default selection")
    ap.add_argument("--T", type=float, default=T_END, help="simulated time (profiling runs)")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 and FWI side runs")
    ap.add_argument("--n3d", type=int, default=400, help="edge of the 3D cube (side run)")
    ap.add_argument("--select", default=None, metavar="METHOD,M,K",
                    help="with --no-search: integrator (faber, hork, hork-horner, krylov, krylov-wQ, "
                         "rk32, rk44, leapfrog, leapfrog-difference), m and step in leap-frog steps "
                         f"(default {','.join(map(str, DEFAULT_SELECTION))})")
    ap.add_argument("--variant", type=int, default=-1,
                    help="FP32 stencil-pass variant (0..14; -1: autotune at first use)")
    ap.add_argument("--case", default="full", choices=["full", "small", "medium", "cube", "signal", "oracle", "fwi"],
                    help="small / medium: the 1001x501 model with 4 / 16 shots (profiling); "
                         "cube: only the 3D side run (--n3d, --check3d); signal: only the "
                         "single-signal experiment of Sec. 4 (FP64, 10 m against 2.5 m); oracle: "
                         "the FP64 oracle run in full on the host cores (no GPU); fwi: only the FWI "
                         "gradient side runs (HORK and Krylov on the 16-shot FWI workload)")
    ap.add_argument("--check3d", type=int, default=0,
                    help="edge of the 3D accuracy cube of a Delta-t_max search (0: time the "
                         "settings found by that search on a 96^3 cube, and check their error "
                         "on a 64^3 cube; -1: time them without the check, for profiling)")
    ap.add_argument("--detail-out", default=None, metavar="PATH",
                    help="also write every side run in full to this JSON file")
    ap.add_argument("--cpu-procs", type=int, default=0,
                    help="oracle processes of the CPU baseline (0: one per host core)")
    return ap.parse_args(argv)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def finite_or_none(obj):
    """A copy of ``obj`` (dicts, lists, tuples, numbers, strings) with every non-finite float
    replaced by None and numpy scalars turned into Python numbers."""
    if isinstance(obj, dict):
        return {str(k): finite_or_none(v) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [finite_or_none(v) for v in obj]
    if isinstance(obj, bool) or obj is None or isinstance(obj, str):
        return obj
    if hasattr(obj, "item") and not isinstance(obj, (int, float)):
        obj = obj.item()                                  # numpy scalar
    if isinstance(obj, float):
        return obj if math.isfinite(obj) else None
    if isinstance(obj, int):
        return obj
    return str(obj)


def json_line(obj):
    """One line of strict JSON (no NaN or Infinity tokens)."""
    return json.dumps(finite_or_none(obj), allow_nan=False, separators=(", ", ": "))


# ------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------------- helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


TMA_SOURCE = os.path.join(ROOT, "paper_2401_16322_gb300", "csrc", "kernels_tma.cu")


def tma_kernel_name(variant):
    """The 2D TMA kernel a variant runs: variants 7 and up use the column-pair consumers."""
    return "stage_tma_x2_kernel" if variant >= 7 else "stage_tma_kernel"


def ncu_traffic_per_point(method, variant):
    """DRAM bytes per grid point of one steady-state stencil pass of ``method`` (a Faber
    degree j >= 2 or a HORK pass after the first) from the committed ncu summary of the
    kernel the variant runs, or None when there is none or the TMA kernel source changed
    since the capture."""
    import hashlib
    name = {"hork": "hork_low_storage", "hork-horner": "hork_horner"}.get(method, method)
    summary = os.path.join(ROOT, "profiles", f"{tma_kernel_name(variant)}_{name}_1001x501x16.md")
    try:
        with open(TMA_SOURCE, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        vals = {}
        with open(summary) as f:
            for line in f:
                if ":" in line and line.startswith("- "):
                    k, v = line[2:].split(":", 1)
                    vals[k.strip()] = v.strip().strip("`")
        if vals.get("kernels_tma.cu sha256") != sha:
            return None
        return float(vals["dram bytes per grid point per pass"])
    except Exception:
        return None


def pass_words(method, m):
    """Algorithmic FP32 words per grid point of each fused stencil pass of one step
    (reads + writes; c^2 counted once per pass)."""
    if method == "faber":
        return [13] + [21] * (m - 1) if m >= 2 else [13]
    if method == "hork-horner":
        return [9] + [13] * (m - 1)      # V_m: X, c^2 -> Y; then V_{j+1}, c^2, V_0 -> V_j
    if method == "hork":
        return [13] + [17] * (m - 1) if m >= 2 else [9]
    if method == "rk32":
        return [13, 13, 13]
    if method == "rk44":
        return [17, 21, 21, 13]
    if method.startswith("krylov"):
        return [13] * m     # x (4) + c^2 (1) + y (4) + dot partner (4)
    if method == "leapfrog":
        return [10]
    if method == "leapfrog-difference":
        return [11]      # u, w_x, w_y (halo), c^2, w^{n-1}, d^n -> u, w_x, w_y, d
    raise ValueError(method)


def _oracle_worker(task):
    """One oracle process: steps of ``method`` on one shot of one model until ``budget_s``
    seconds have passed.  Returns (grid-point-steps, seconds, steps)."""
    (nx, ny, dx, order, pml, beta0, fs, c, sx, sy, f_peak, t0, method, m, dt, t_start,
     budget_s, ellipse) = task
    from oracle.model import Model as OModel
    from oracle.simulate import run
    from oracle.source import PointSource
    om = OModel(nx, ny, dx, order, pml, beta0, fs, c)
    src = PointSource(om, sx, sy, f_peak, t0, 1.0, p=12)
    U = om.zeros_state()
    t0w = time.perf_counter()
    nsteps = 0
    while True:
        U, _ = run(om, method, dt, 1, src=src, m=m, U0=U, t0=t_start + nsteps * dt,
                   faber_params=ellipse)
        nsteps += 1
        if time.perf_counter() - t0w >= budget_s:
            break
    return nsteps * nx * ny, time.perf_counter() - t0w, nsteps


class OracleSampler:
    """The FP64 CPU oracle timed on the host cores: ``procs`` processes (spawned, one
    numpy thread each) each step one shot of the 458 x 229 model of the batched workload for
    a bounded time, on different shot positions; the rate is the grid-point-steps of all of
    them over the wall time of the sample.  The oracle runs as it stands; the processes only
    run independent shots side by side, as the shots of the workload are independent."""

    def __init__(self, procs=0):
        import multiprocessing as mp
        self.procs = procs if procs > 0 else (os.cpu_count() or 1)
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        self.pool = mp.get_context("spawn").Pool(self.procs)
        self.pool.map(abs, range(self.procs))            # start every process before timing

    def sample(self, workloads, method, m, dt, budget_s):
        """(seconds per grid-point-step of the whole host, description, cores, wall seconds,
        grid-point-steps sampled)."""
        from oracle.faber import ellipse_params
        from paper_2401_16322_gb300.tts import pml_beta0
        from paper_2401_16322_gb300.workloads import t0_for
        w = workloads[4]                                   # 458 x 229 model
        c_max = max(float(x.c.max()) for x in workloads)
        beta0 = pml_beta0(c_max, w.pml, w.dx)
        ell = ellipse_params(c_max, beta0, w.dx, w.order, free_surface=w.free_surface)
        # the oracle evaluates HORK in the paper's stages and Krylov with full orthogonalisation
        om_method = {"hork-horner": "hork", "leapfrog-difference": "leapfrog"}.get(
            method, "krylov" if method.startswith("krylov") else method)
        tasks = []
        for q in range(self.procs):
            sx = (40 + (w.nx - 80) * (q + 0.5) / self.procs) * w.dx
            tasks.append((w.nx, w.ny, w.dx, w.order, w.pml, beta0, w.free_surface, w.c, sx,
                          w.shots[0].sy, w.f_peak, t0_for(w.f_peak), om_method, m, dt, 0.3,
                          budget_s, ell))
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, tasks, chunksize=1)
        wall = time.perf_counter() - t0
        pts = sum(r[0] for r in res)
        steps = sum(r[2] for r in res)
        desc = (f"oracle {om_method}(m={m}, dt={dt * 1e3:.3f} ms) FP64 on {self.procs} processes, "
                f"{steps} steps of {self.procs} shots of the {w.nx}x{w.ny} model in {wall:.1f} s "
                f"wall, scaled by grid-point-steps to the whole batch")
        return wall / pts, desc, self.procs, wall, pts

    def close(self):
        self.pool.terminate()
        self.pool.join()


def batch_points(workloads):
    return sum(w.nx * w.ny * len(w.shots) for w in workloads)


def fp64_single_shot_estimate(wl, method, m, dt, nsteps, c_max, steps_sample=3):
    """The plain FP64 single-shot form of the selected method: every model alone, one shot,
    timed for a few steps and scaled to all shots and steps (seconds)."""
    import torch
    from paper_2401_16322_gb300.tts import base_method, build_models, common_ellipse
    from paper_2401_16322_gb300.workloads import Workload
    total = 0.0
    for w in wl:
        one = Workload(w.name, w.nx, w.ny, w.dx, w.order, w.pml, w.free_surface, w.c, w.shots[:1],
                       w.f_peak, w.T)
        md = build_models([one], "f64", p=12, c_max=c_max)[0]
        common_ellipse([md], c_max)
        method = base_method([md], method)
        md.ensure_workspace(method, m)
        md.step(method, 0.25, dt, m, 1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        md.step(method, 0.25, dt, m, steps_sample)
        e1.record()
        md.sync()
        total += e0.elapsed_time(e1) / steps_sample * nsteps * len(w.shots) * 1e-3
        md.close()
    return {"time_to_solution_s": total, "sample": f"{steps_sample} FP64 steps of one shot per "
            "model, scaled to every shot and step, one shot per launch"}


def fwi_gradient_step(method, m, dt_over_cfl):
    """FWI gradient (forward + adjoint) on the 401 x 201, 16-shot, 200-receiver workload,
    FP32, with the given integrator at its m and step ratio; every state checkpointed.  The
    polynomial steps take their exact discrete adjoints; Krylov takes the adjoint of the
    step's exponential, because the exact adjoint of a Krylov step of dimension 20 at 8 x
    the leap-frog step is ill-conditioned over this run (its cotangent grows without bound
    while the source is still silent); tests/test_gpu_fwi.py checks both against central
    differences on this workload.  The Krylov forward keeps every step's four dense states
    (ewv_step_krylov_dense), so its adjoint runs no forward Arnoldi; the recomputing form is
    timed beside it."""
    import numpy as np
    import torch
    from paper_2401_16322_gb300.fwi import FaberFWI
    from paper_2401_16322_gb300.tts import base_method, build_models, common_ellipse, leapfrog_step
    from paper_2401_16322_gb300.workloads import config_fwi, smooth_gradient_with_anomalies
    if method not in ("faber", "hork", "hork-horner", "krylov"):
        return None
    w = config_fwi()
    c_max = float(w.c.max()) * 1.05
    dt = dt_over_cfl * leapfrog_step(c_max, w.dx, w.order)
    nsteps = int(round(w.T / dt))
    md = build_models([w], "f32", p=12, c_max=c_max)[0]
    common_ellipse([md], c_max)
    if method == "krylov":
        md.set_krylov_adjoint("exponential")
    c_init = smooth_gradient_with_anomalies(w.nx, w.ny, 0, dx=w.dx, amps=())

    def timed(dense):
        fwi = FaberFWI(md, dt, m, nsteps, len(w.shots[0].rec), method=base_method([md], method),
                       dense_states=dense)
        d_obs = fwi.forward(w.c ** 2)
        fwi.backward(fwi.forward(c_init ** 2) - d_obs)     # warm-up: workspaces, graphs, tuning
        torch.cuda.synchronize()
        e0, em, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        seis = fwi.forward(c_init ** 2)
        em.record()
        grad = fwi.backward(seis - d_obs)
        e1.record()
        torch.cuda.synchronize()
        out = {"seconds": e0.elapsed_time(e1) * 1e-3, "forward_s": e0.elapsed_time(em) * 1e-3,
               "backward_s": em.elapsed_time(e1) * 1e-3, "stored_bytes": fwi.stored_bytes(),
               "gradient_finite": bool(torch.isfinite(grad).all())}
        del fwi
        return out

    res = timed(method == "krylov")
    res.update({"method": method, "nsteps": nsteps,
                "adjoint": ("adjoint of the step's exponential from the forward's dense states "
                            "(FD-checked to 2e-3 on this workload)"
                            if method == "krylov" else "exact discrete adjoint"),
                "dt_ms": dt * 1e3, "m": m, "shots": len(w.shots), "grid": f"{w.nx}x{w.ny}"})
    if method == "krylov":
        res["recomputing_forward_arnoldi"] = timed(False)
    md.close()
    return res


# Delta-t_max scan of the 3D side run: (method, m values, step multiples, largest first)
SCAN3D = (("faber", (30, 40, 50, 60), tuple(range(24, 1, -1))),
          ("hork", (12, 16, 24), tuple(range(12, 0, -1))),
          ("hork-horner", (12, 16, 24), tuple(range(12, 0, -1))),
          ("krylov", (20,), tuple(range(24, 1, -1))))
LEAPFROG3D_DIVISORS = (1, 2, 3, 4, 6, 8)
# settings of the last 3D Delta-t_max search (method, m, step in 3D leap-frog steps)
FIXED3D = (("hork-horner", 16, 3.0), ("faber", 60, 12.0), ("krylov", 20, 8.0), ("leapfrog", 1, 0.5))


def config5_3d(n=400, check_n=0, target=TARGET):
    """The three-dimensional workload (n^3 layered cube, 8th order, free surface, 30-point ABC,
    Ricker 10 Hz, T = 1 s; FP32).

    1. Delta-t_max search on a check_n^3 cube of the same construction over T = 0.5 s: for
       every (method, m) the largest multiple of the 3D leap-frog step whose seismogram is
       within the target of an FP64 reference (Faber 30 at the leap-frog step); leap-frog at
       1 .. 1/8 of its step.
    2. Time per step of each passing (method, m) at its Delta-t_max on the n^3 cube, time to
       T, and the roofline of the 3D TMA pass (Faber).
    check_n = 0 skips the search: the settings of FIXED3D (found by an earlier search) are
    checked for error and stability on a 64^3 cube of the same construction, then timed.
    """
    import numpy as np
    import torch
    from paper_2401_16322_gb300 import Model
    from paper_2401_16322_gb300.tts import (base_method, dt_max_scan, leapfrog_step, pml_beta0,
                                            rel_l2_common)
    from paper_2401_16322_gb300.workloads import config_3d, t0_for
    c_max = 4500.0

    def build(w, prec, p=12):
        b0 = pml_beta0(c_max, w.pml, w.dx)
        md = Model(w.n, w.n, w.dx, w.order, w.pml, b0, w.free_surface, precision=prec, p=p,
                   max_receivers=len(w.rec), nz=w.n)
        md.set_velocity(w.c)
        md.set_source_receivers3d(0, *w.src, w.f_peak, t0_for(w.f_peak), 1.0, w.rec)
        return md

    def simulate(md, method, m, dt, T):
        nsteps = int(round(T / dt))
        md.bind_seismogram(nsteps)
        md.reset_state()
        md.step(base_method([md], method), 0.0, dt, m, nsteps)
        md.sync()
        return md.seismogram(0, md.max_receivers, nsteps)

    out = {"workload": f"{n}^3 layered, dx 10 m, 8th order, free surface, 30-pt ABC, Ricker 10 Hz, "
                       "T 1 s, FP32", "target": target, "candidates": [],
           "pml": "auxiliary-field PML (psi_t = u), exact reduction to Eq. 1"}
    found = []          # (method, m, k, err); k < 1: leap-frog divisor 1/k
    t_search = time.perf_counter()
    n_check = check_n if check_n > 0 else 64
    wc = config_3d(n_check, pml=min(20, n_check // 4), T=0.5)
    dt3 = leapfrog_step(c_max, wc.dx, dims=3)
    ref_md = build(wc, "f64", p=20) if check_n >= 0 else None
    ref = simulate(ref_md, "faber", 30, dt3, wc.T) if ref_md is not None else None
    log(f"3D reference {time.perf_counter() - t_search:.1f} s")
    cmd = build(wc, "f32")

    from paper_2401_16322_gb300 import Batch
    from paper_2401_16322_gb300.tts import NOISE_GROWTH, POLYNOMIAL, noise_growth
    cbatch = Batch([cmd])
    t_quiet = wc.T + 20.0 / wc.f_peak + t0_for(wc.f_peak)

    def err_of(md, method, m, dt):
        try:
            err = rel_l2_common(simulate(md, method, m, dt, wc.T), dt, ref, dt3)
            if err <= target and method in POLYNOMIAL and md is cmd:
                # the stability check of the 2D search (white noise, source silent)
                growth = noise_growth([cmd], cbatch, method, m, dt, t_quiet)
                if not growth <= NOISE_GROWTH:
                    log(f"3D {method} m={m} dt={dt * 1e3:.3f} ms: noise grows {growth:.3g} x")
                    return float("inf")
            return err
        except Exception as e:       # e.g. a non-finite Arnoldi step
            log(f"3D {method} m={m} dt={dt * 1e3:.3f} ms: {e}")
            return float("inf")

    if check_n < 0:
        # profiling runs: time the settings of FIXED3D without the check cube
        found.extend((method, m, float(k), float("nan")) for method, m, k in FIXED3D)
        out["error_check"] = None
    elif check_n > 0:
        for method, ms, ks in SCAN3D:
            for m in ms:
                errs = {}
                k, _ = dt_max_scan(ks, lambda k: errs.setdefault(k, err_of(cmd, method, m, k * dt3)),
                                   target)
                if k is not None:
                    found.append((method, m, float(k), errs[k]))
                log(f"3D {method} m={m}: dt_max = " + (f"{k} x leap-frog step" if k else "none")
                    + f" ({time.perf_counter() - t_search:.1f} s)")
        for prec, md in (("f32", cmd), ("f64", ref_md)):
            errs = {}
            k, _ = dt_max_scan(LEAPFROG3D_DIVISORS,
                               lambda k: errs.setdefault(k, err_of(md, "leapfrog", 1, dt3 / k)), target)
            if k is not None:
                found.append(("leapfrog" if prec == "f32" else "leapfrog_f64", 1, 1.0 / k, errs[k]))
        out["error_check"] = f"{check_n}^3 cube, T 0.5 s, FP64 Faber 30 at the 3D leap-frog step"
    else:
        # the settings an earlier search found (FIXED3D), each checked for error and
        # stability on a 64^3 cube
        for method, m, k in FIXED3D:
            dt = k * dt3
            err = err_of(cmd, method, m, dt)
            if err <= target:
                found.append((method, m, float(k), err))
            else:
                log(f"3D {method} m={m} at {k} x: error {err:.3e} above the target")
        out["error_check"] = "64^3 cube, T 0.5 s, FP64 Faber 30 at the 3D leap-frog step"
    if ref_md is not None:
        ref_md.close()
    cbatch.close()
    cmd.close()
    out["search_s"] = time.perf_counter() - t_search
    # timing on the full cube
    w = config_3d(n)
    dt3 = leapfrog_step(c_max, w.dx, dims=3)
    t_live = t0_for(w.f_peak)
    peak, peak_kind = measured_peaks()
    md = build(w, "f32")
    md64 = None
    for method, m, k, err in found:
        dt = k * dt3
        prec = "f32"
        dev = md
        if method == "leapfrog_f64":
            if md64 is None:
                md.close()
                md = None
                md64 = build(w, "f64")
            dev, prec, method = md64, "f64", "leapfrog"
        bm = base_method([dev], method)
        dev.ensure_workspace(bm, m)
        dev.reset_state()
        try:
            dev.step(bm, t_live - 2 * dt, dt, m, 2)
            torch.cuda.synchronize()
            dev.enable_kernel_timing(True)
            dev.kernel_timing()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ns = 4
            e0.record()
            dev.step(bm, t_live, dt, m, ns)
            e1.record()
            dev.sync()
            kms, kn = dev.kernel_timing()
            dev.enable_kernel_timing(False)
        except Exception as e:
            log(f"3D {method} m={m} at {k} x fails on the {n}^3 cube: {e}")
            continue
        step_ms = e0.elapsed_time(e1) / ns
        nsteps = int(round(w.T / dt))
        cand = {"method": method, "precision": prec, "m": m, "dt_over_leapfrog_step": k,
                "dt_ms": dt * 1e3, "ms_per_step": step_ms, "nsteps_to_T": nsteps,
                "time_to_T_s": step_ms * nsteps * 1e-3,
                "grid_point_updates_per_s": n ** 3 / (step_ms * 1e-3),
                "seismo_rel_err_vs_fp64": err}
        if method in ("faber", "hork-horner") and kn and prec == "f32":
            words = pass_words3d(method, m)
            per_launch = sum(words) * 4.0 * n ** 3 / len(words)
            avg = kms / kn * 1e-3
            cand["roofline"] = {"bound": "hbm", "kernel": "stage_tma3d_kernel (FP32)",
                                "achieved": per_launch / avg / 1e9, "peak": peak, "unit": "GB/s",
                                "frac": per_launch / avg / 1e9 / peak, "peak_kind": peak_kind,
                                "avg_launch_us": avg * 1e6, "alg_bytes_per_launch": per_launch}
        out["candidates"].append(cand)
        log(f"3D {method} ({prec}) m={m} at {k:.3g} x: {step_ms:.2f} ms/step, {nsteps} steps, "
            f"{cand['time_to_T_s']:.2f} s, err {err:.3e}")
    # the 3D pass of each fused integrator timed on its own, whether or not its step was
    # selected: 4 steps of Faber 40 and of HORK 16 in Horner form at 2 x the 3D leap-frog step
    if md is not None:
        out["pass_rooflines"] = {}
        for method, m in (("faber", 40), ("hork-horner", 16)):
            try:
                dt = 2.0 * dt3
                bm = base_method([md], method)
                md.ensure_workspace(bm, m)
                md.reset_state()
                md.step(bm, t_live - 2 * dt, dt, m, 2)
                torch.cuda.synchronize()
                md.enable_kernel_timing(True)
                md.kernel_timing()
                md.step(bm, t_live, dt, m, 4)
                md.sync()
                kms, kn = md.kernel_timing()
                md.enable_kernel_timing(False)
                words = pass_words3d(method, m)
                per_launch = sum(words) * 4.0 * n ** 3 / len(words)
                avg = kms / kn * 1e-3
                out["pass_rooflines"][method] = {
                    "m": m, "bound": "hbm", "kernel": "stage_tma3d_kernel (FP32)",
                    "achieved": per_launch / avg / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": per_launch / avg / 1e9 / peak, "peak_kind": peak_kind,
                    "avg_launch_us": avg * 1e6, "alg_bytes_per_launch": per_launch}
                log(f"3D {method} pass: {avg * 1e6:.1f} us, "
                    f"{per_launch / avg / 1e9 / peak:.3f} of the {peak_kind} copy peak")
            except Exception as e:
                md.enable_kernel_timing(False)
                log(f"3D {method} pass timing failed: {e}")
    for d in (md, md64):
        if d is not None:
            d.close()
    exp = [c for c in out["candidates"] if c["method"] != "leapfrog"]
    if exp:
        out["selected"] = min(exp, key=lambda c: c["time_to_T_s"])
    fr = [c["roofline"]["frac"] for c in out["candidates"] if "roofline" in c]
    out["roofline_frac"] = max(fr) if fr else None
    lf = [c for c in out["candidates"] if c["method"] == "leapfrog"]
    if lf:
        out["leapfrog_best"] = min(lf, key=lambda c: c["time_to_T_s"])
    return out


def pass_words3d(method, m):
    """Algorithmic FP32 words per point of each 3D stencil pass (six fields: u, v, w_x, w_y,
    w_z, psi; c^2 once)."""
    if method == "faber":
        return [19] + [31] * (m - 1) if m >= 2 else [19]
    if method == "hork-horner":
        return [13] + [19] * (m - 1)
    if method == "hork":
        return [19] + [25] * (m - 1) if m >= 2 else [13]
    raise ValueError(method)


def config1_fp64_study():
    """The small homogeneous case (101 x 101, dx 10 m, 2000 m/s, 4th order, 20-point ABC,
    Ricker 15 Hz at the centre, 50 receivers, T 0.5 s) in FP64: Delta-t_max of Faber, HORK
    and Krylov against an FP64 reference (Faber 30 at the leap-frog step) and leap-frog at
    1 .. 1/32 of its step, each candidate's error and its time to T on the GPU.  Every
    evaluated (method, m, step) is listed, so the error-versus-step curves can be drawn."""
    from paper_2401_16322_gb300 import Batch
    from paper_2401_16322_gb300.tts import build_models, run_study
    from paper_2401_16322_gb300.workloads import config_homogeneous_small
    wl = [config_homogeneous_small()]
    plan = (("faber", (10, 20, 30, 40), tuple(range(16, 0, -1))),
            ("hork", (8, 12, 16), tuple(range(8, 0, -1))),
            ("krylov", (10, 20), tuple(range(16, 0, -1))))
    models = build_models(wl, "f64", p=12)
    batch = Batch(models)
    st = run_study(wl, [(0, 0)], wl[0].T, plan=plan, full_batch=batch, full_models=models,
                   precision="f64", log=lambda *a: None)
    batch.close()
    for md in models:
        md.close()
    cand = [{"method": c.method, "m": c.m, "dt_ms": round(c.dt * 1e3, 5),
             "seismo_rel_err": c.err, "time_to_T_s": c.cost_s} for c in st.candidates]
    sel = st.selected
    return {"workload": "homogeneous 101x101, 4th order, FP64, T 0.5 s",
            "leapfrog_step_ms": st.dt_cfl * 1e3,
            "selected": ({"method": sel.method, "m": sel.m, "dt_ms": sel.dt * 1e3,
                          "seismo_rel_err": sel.err, "time_to_T_s": sel.cost_s} if sel else None),
            "leapfrog": ({"dt_ms": st.leapfrog.dt * 1e3, "seismo_rel_err": st.leapfrog.err,
                          "time_to_T_s": st.leapfrog.cost_s} if st.leapfrog else None),
            "evaluated": cand, "search_s": st.seconds}


def max_over_ranks(value, dist=None, device="cuda"):
    """The largest value over the ranks (the slowest rank sets a step's time); the value itself
    on a single process."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------- full oracle runs
def _oracle_full_worker(task):
    """One whole oracle simulation of one shot (no time budget): (seconds, steps, points)."""
    (nx, ny, dx, order, pml, beta0, fs, c, sx, sy, f_peak, t0, method, m, dt, nsteps, ellipse) = task
    from oracle.model import Model as OModel
    from oracle.simulate import run
    from oracle.source import PointSource
    om = OModel(nx, ny, dx, order, pml, beta0, fs, c)
    src = PointSource(om, sx, sy, f_peak, t0, 1.0, p=12)
    t_start = time.perf_counter()
    run(om, method, dt, nsteps, src=src, m=m, t0=0.0, faber_params=ellipse)
    return time.perf_counter() - t_start, nsteps, nx * ny


def oracle_full_runs(procs=0):
    """The FP64 oracle run in full (not sampled) on the small homogeneous case, the 601 x 301
    model and the 16-shot FWI model, with the settings the GPU runs use: one process for a
    single shot, and the 16 shots on one process (measured on one shot, times 16) and on every
    host core (shots in parallel, measured)."""
    import multiprocessing as mp
    import platform
    from oracle.faber import ellipse_params
    from paper_2401_16322_gb300.tts import leapfrog_step, pml_beta0
    from paper_2401_16322_gb300.workloads import (config_fwi, config_homogeneous_small,
                                                  config_layered_601x301, t0_for)
    procs = procs if procs > 0 else (os.cpu_count() or 1)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"

    def tasks(w, method, m, k, shots, beta0=None, dims_c=None):
        c_max = float(w.c.max())
        b0 = pml_beta0(c_max, w.pml, w.dx) if beta0 is None else beta0
        dt = k * leapfrog_step(c_max, w.dx, w.order)
        nsteps = int(round(w.T / dt))
        ell = ellipse_params(c_max, b0, w.dx, w.order, free_surface=w.free_surface)
        return [(w.nx, w.ny, w.dx, w.order, w.pml, b0, w.free_surface, w.c, s.sx, s.sy, w.f_peak,
                 t0_for(w.f_peak), method, m, dt, nsteps, ell) for s in shots], dt, nsteps

    out = {"cpu": platform.processor() or platform.machine(), "cores": procs, "runs": []}
    w1 = config_homogeneous_small()
    w2 = config_layered_601x301()
    w4 = config_fwi()
    pool = mp.get_context("spawn").Pool(procs)
    pool.map(abs, range(procs))
    for name, w, method, m, k in (("homogeneous 101x101, 4th order", w1, "hork", 12, 2.0),
                                  ("layered 601x301", w2, "hork", 20, 4.0),
                                  ("FWI model 401x201, one shot", w4, "krylov", 20, 8.0)):
        tk, dt, nsteps = tasks(w, method, m, k, w.shots[:1])
        sec, _, pts = pool.apply(_oracle_full_worker, (tk[0],))
        out["runs"].append({"workload": name, "method": method, "m": m, "dt_ms": dt * 1e3,
                            "nsteps": nsteps, "processes": 1, "seconds": sec,
                            "grid_point_steps_per_s": pts * nsteps / sec})
        log(f"oracle {name}: {sec:.1f} s")
    tk, dt, nsteps = tasks(w4, "krylov", 20, 8.0, w4.shots)
    t_start = time.perf_counter()
    res = pool.map(_oracle_full_worker, tk, chunksize=1)
    wall = time.perf_counter() - t_start
    one = out["runs"][-1]["seconds"]
    out["runs"].append({"workload": "FWI model 401x201, 16 shots (forward)", "method": "krylov", "m": 20,
                        "dt_ms": dt * 1e3, "nsteps": nsteps, "processes": procs, "seconds": wall,
                        "one_process_seconds_est": 16 * one,
                        "grid_point_steps_per_s": sum(r[2] * r[1] for r in res) / wall})
    pool.terminate()
    pool.join()
    return out


# ------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2401_16322_gb300.tts import leapfrog_step
    from paper_2401_16322_gb300.workloads import config_batched
    sampler = OracleSampler(args.cpu_procs)
    wl = config_batched()
    c_max = max(float(w.c.max()) for w in wl)
    dt_cfl = leapfrog_step(c_max, wl[0].dx, wl[0].order)
    method, m, k = DEFAULT_SELECTION
    dt = k * dt_cfl
    nsteps = int(round(T_END / dt))
    pts = batch_points(wl)
    budget = max(1.0, min(args.cpu_sample_s, 60.0 / max(1, args.steps + args.warmup)))
    vals, walls, sampled = [], [], 0
    for it in range(args.warmup + args.steps):
        pps, desc, cores, wall, npts = sampler.sample(wl, method, m, dt, budget)
        if it >= args.warmup:
            vals.append(pps * pts * nsteps)
            walls.append(wall)
            sampled += npts
    sampler.close()
    v = statistics.mean(vals)
    # a step of this arm is one bounded sample of the oracle (its wall time is ms_per_step);
    # the value is the whole batch's time to solution at the sampled rate (extrapolated)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(walls) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "method": method, "m": m, "dt_ms": dt * 1e3,
                       "T_s": T_END, "grid_points": pts, "nsteps": nsteps},
            "extrapolated": True,
            "sampled_grid_point_steps": sampled, "sample_wall_s": sum(walls),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc, "extrapolated": True},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json_line(line), flush=True)
    return 0


# ------------------------------------------------------------------------- our arm
def check_problems(wl, models, method, m, dt, nsteps, c_max, dt_cfl, study, target):
    """Seismogram error of the selected setting on CHECK_PROBLEMS (17 of the 72 problems),
    taken from the last simulation of the timed region, against an FP64 Faber reference of
    degree 60 at dt / q (q the smallest integer with dt / q <= 6 leap-frog steps; the Faber
    coefficients beyond degree 60 are below 1e-15 there), or of degree 30 at the leap-frog
    step when dt is smaller.  On the three problems of the search the reference is compared
    with the search's own FP64 reference."""
    from paper_2401_16322_gb300 import Batch
    from paper_2401_16322_gb300.tts import (build_models, common_ellipse, rel_l2_common,
                                            sampled_workloads, simulate)
    t0 = time.perf_counter()
    got = []
    for wi, si in CHECK_PROBLEMS:
        md = models[wi]
        nrec = len(wl[wi].shots[si].rec)
        s = md.seismo.view(md.nshots, md.capacity, md.max_receivers)[si, :nsteps, :nrec]
        got.append(s.double().cpu().numpy())
    if dt >= dt_cfl * (1 - 1e-9):
        q = max(1, math.ceil(dt / (6.0 * dt_cfl) - 1e-9))
        dt_ref, m_ref = dt / q, 60
    else:
        dt_ref, m_ref = dt_cfl, 30
    sw = sampled_workloads(wl, CHECK_PROBLEMS)
    ref_models = build_models(sw, "f64", p=20, c_max=c_max)
    common_ellipse(ref_models, c_max)
    rb = Batch(ref_models)
    n_ref = simulate(ref_models, rb, "faber", m_ref, dt_ref, nsteps * dt)
    errs, cross = [], []
    for (wi, si), md, w, g in zip(CHECK_PROBLEMS, ref_models, sw, got):
        ref = md.seismogram(0, len(w.shots[0].rec), n_ref)
        errs.append(rel_l2_common(g, dt, ref, dt_ref))
        if study is not None and (wi, si) in PICKS:
            sref = study.refs[PICKS.index((wi, si))]
            cross.append(rel_l2_common(ref, dt_ref, sref, study.dt_ref))
    rb.close()
    for md in ref_models:
        md.close()
    worst = int(max(range(len(errs)), key=lambda i: errs[i] if math.isfinite(errs[i]) else 1e300))
    return {"problems": len(errs), "of": sum(len(w.shots) for w in wl),
            "max_rel_err": max(errs) if all(math.isfinite(e) for e in errs) else float("inf"),
            "worst_problem": list(CHECK_PROBLEMS[worst]),
            "all_within_target": all(e <= target for e in errs),
            "reference": f"FP64 faber m={m_ref} dt={dt_ref * 1e3:.4f} ms",
            "reference_vs_search_reference": max(cross) if cross else None,
            "per_problem": [[wi, si, e] for (wi, si), e in zip(CHECK_PROBLEMS, errs)],
            "seconds": time.perf_counter() - t0}


def max_amplification(method, m, dt, dt_cfl, ellipse):
    """Largest |R(i omega dt)| of a polynomial integrator over 0 < omega <= omega_top, where
    omega_top = 2 / (leap-frog step) = c_max sqrt(2 |S2|) / dx is the top of the undamped
    interior spectrum (above 1: modes there grow by that factor per step)."""
    import numpy as np
    from paper_2401_16322_gb300.analysis import amplification
    if method not in ("faber", "hork", "hork-horner", "rk32", "rk44"):
        return None
    om = np.linspace(0.0, 2.0 / dt_cfl, 4001)[1:]
    return float(np.max(np.abs(amplification(method, m, om, dt, ellipse))))


def run_ours(args):
    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2401_16322_gb300 import Batch
    from paper_2401_16322_gb300.tts import (build_models, common_ellipse, leapfrog_step, run_study,
                                            simulate)
    from paper_2401_16322_gb300.workloads import config_batched

    t_run = time.perf_counter()
    if args.case == "full":
        wl = config_batched()
    else:
        wl = config_batched(nshots=4 if args.case == "small" else 16)[:1]
    T_run = args.T
    c_max = max(float(w.c.max()) for w in wl)
    dt_cfl = leapfrog_step(c_max, wl[0].dx, wl[0].order)
    pts = batch_points(wl)
    t_setup = time.perf_counter()
    models = build_models(wl, "f32", p=12, c_max=c_max)
    ellipse = common_ellipse(models, c_max)
    batch = Batch(models)
    if args.variant >= 0:
        batch.set_kernel_variant(args.variant)
    log(f"setup {time.perf_counter() - t_setup:.1f} s, {pts} grid points, dt_cfl {dt_cfl * 1e3:.4f} ms")

    method, m, k = DEFAULT_SELECTION
    if args.select:
        sm, sk, skk = args.select.split(",")
        method, m, k = sm, int(sk), float(skk)
    study = None
    growth = float("nan")
    if not args.no_search and args.case == "full":
        models64 = build_models(wl, "f64", p=12, c_max=c_max)   # FP64 leap-frog timing
        study = run_study(wl, PICKS, T_run, target=args.target, full_batch=batch, full_models=models,
                          full_models_f64=models64, log=log if rank == 0 else (lambda *a: None),
                          self_check=True)
        for md in models64:
            md.close()
        del models64
        if study.selected is not None:
            method, m, dt = study.selected.method, study.selected.m, study.selected.dt
            growth = study.selected.growth
        else:
            dt = k * dt_cfl
        seismo_err = study.selected.err if study.selected else float("nan")
    else:
        dt = k * dt_cfl
        seismo_err = float("nan")
    nsteps = int(round(T_run / dt))
    log(f"selected {method} m={m} dt={dt * 1e3:.4f} ms ({nsteps} steps), sampled error {seismo_err:.3e} "
        f"({time.perf_counter() - t_run:.0f} s into the run)")

    def one_solution():
        simulate(models, batch, method, m, dt, T_run)

    # ---- timed region: K whole simulations, no per-pass instrumentation
    batch.enable_kernel_timing(False)
    for _ in range(args.warmup):
        one_solution()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = batch.launch_count()
    clk = ClockSampler(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        one_solution()
    e1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = clk.stop()
    elapsed_ms = e0.elapsed_time(e1)
    launches = batch.launch_count() - launches0
    ms_per_step = elapsed_ms / args.steps
    ms_per_step = max_over_ranks(ms_per_step, dist)
    # every problem's seismogram of the last timed simulation is finite
    all_finite = all(bool(torch.isfinite(md.seismo).all()) for md in models)
    log(f"timed: {ms_per_step:.1f} ms per solution ({time.perf_counter() - t_run:.0f} s into the run)")

    # ---- error of the last timed simulation on a spread of problems
    check = None
    if rank == 0 and args.case == "full" and T_run == T_END:
        check = check_problems(wl, models, method, m, dt, nsteps, c_max, dt_cfl, study, args.target)
        log(f"error on {check['problems']} problems: max {check['max_rel_err']:.3e} "
            f"({check['seconds']:.1f} s)")

    # ---- roofline: one more simulation with CUDA events around every stencil pass
    batch.enable_kernel_timing(True)
    batch.kernel_timing()
    one_solution()
    torch.cuda.synchronize()
    kern_ms, kern_n = batch.kernel_timing()
    batch.enable_kernel_timing(False)
    words = pass_words(method, m)
    alg_bytes_per_step = sum(words) * 4.0 * pts
    per_launch_bytes = alg_bytes_per_step / len(words)
    avg_launch_ms = kern_ms / max(kern_n, 1)
    achieved = per_launch_bytes / (avg_launch_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()

    # ---- e2e through the public API: velocity models in, every seismogram out, per solution
    vel_host = [np.ascontiguousarray(w.c) for w in wl]
    h2d = sum(v.nbytes for v in vel_host)
    pinned = [torch.empty(md.seismo.numel(), dtype=md.seismo.dtype, pin_memory=True) for md in models]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(args.steps):
        for md, v in zip(models, vel_host):
            md.set_velocity(v)
        simulate(models, batch, method, m, dt, T_run)
        d2h = 0
        for md, buf in zip(models, pinned):
            buf.copy_(md.seismo, non_blocking=True)
            d2h += buf.numel() * buf.element_size()
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = max_over_ranks(e2e_s, dist)
    log(f"e2e: {e2e_s:.3f} s per solution ({time.perf_counter() - t_run:.0f} s into the run)")

    extras = {}
    if rank == 0 and args.case == "full" and not args.no_extras:
        for name, fn in (("fp64_single_shot", lambda: fp64_single_shot_estimate(wl, method, m, dt, nsteps, c_max)),
                         ("fwi_gradient", lambda: fwi_gradient_step(method, m, dt / dt_cfl)),
                         ("fwi_gradient_krylov", lambda: fwi_gradient_step("krylov", 20, 8.0)),
                         ("config5_3d", lambda: config5_3d(args.n3d, args.check3d)),
                         ("config1_fp64", config1_fp64_study)):
            t_x = time.perf_counter()
            try:
                extras[name] = fn()
            except Exception as e:           # a side run never costs the headline
                extras[name] = {"error": f"{type(e).__name__}: {e}"}
            log(f"side run {name}: {time.perf_counter() - t_x:.1f} s")
    if rank == 0 and study is not None:
        # dispersion / dissipation of the fastest passing setting of each method (and of
        # leap-frog at its passing FP64 step) on the undamped spectrum
        from paper_2401_16322_gb300.analysis import report
        best = {}
        for c in study.candidates:
            if c.err <= args.target and not c.method.startswith("krylov") and math.isfinite(c.cost_s):
                if c.method not in best or c.cost_s < best[c.method].cost_s:
                    best[c.method] = c
        if study.leapfrog_f64 is not None:
            best["leapfrog"] = study.leapfrog_f64
        # top of the undamped interior spectrum, c_max sqrt(2 |S2|) / dx = 2 / leap-frog step
        extras["dispersion"] = report([(c.method, c.m, c.dt) for c in best.values()],
                                      wl[0].f_peak, 2.0 / dt_cfl, ellipse)
    if rank == 0:
        sampler = OracleSampler(args.cpu_procs)
        cpu_pps, cpu_desc, cores, _, _ = sampler.sample(config_batched(), method, m, dt, args.cpu_sample_s)
        sampler.close()
        cpu_tts = cpu_pps * pts * nsteps
        lf = study.leapfrog if study else None
        lf64 = study.leapfrog_f64 if study else None

        def brief(c):
            return {"dt_ms": c.dt * 1e3, "seismo_rel_err": c.err, "time_to_solution_s": c.cost_s}

        passing = sorted([c for c in study.candidates if c.err <= args.target and math.isfinite(c.cost_s)],
                         key=lambda c: c.cost_s) if study else []
        best_per_method = {}
        for c in passing:
            best_per_method.setdefault(c.method, c)
        x3 = extras.get("config5_3d") or {}
        f1 = extras.get("config1_fp64") or {}
        fp = extras.get("fwi_gradient") or {}
        fk = extras.get("fwi_gradient_krylov") or {}
        kvar = {k_: v_ for k_, v_ in batch.kernel_variant().items() if k_ != "probe_us"}
        result = {
            "metric": METRIC, "value": ms_per_step / 1e3, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME if args.case == "full" else f"{args.case}: 1001x501, {len(wl[0].shots)} shots",
                       "method": method, "m": m, "dt_ms": dt * 1e3,
                       "dt_over_leapfrog_step": dt / dt_cfl, "nsteps": nsteps, "T_s": T_run,
                       "grid_points": pts, "problems": sum(len(w.shots) for w in wl),
                       "l2": "inputs larger than L2 (state + workspace > 1 GB)",
                       "parallelism": f"replicas x{world}"},
            "seismo_rel_err_search_problems": seismo_err,
            "seismo_rel_err_max_over_checked_problems": check["max_rel_err"] if check else None,
            "checked_problems": ({"count": check["problems"], "of": check["of"],
                                  "all_within_target": check["all_within_target"],
                                  "worst": check["worst_problem"], "reference": check["reference"],
                                  "reference_vs_search_reference": check["reference_vs_search_reference"]}
                                 if check else None),
            "all_seismograms_finite": all_finite,
            "stability": {"noise_growth_per_100_steps": growth, "limit": NOISE_LIMIT(),
                          "noise_problems": study.noise_problems if study else None,
                          "max_amplification_interior": max_amplification(method, m, dt, dt_cfl, ellipse)},
            "grid_point_updates_per_s": pts * nsteps / (ms_per_step / 1e3),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": (tpp * pts if (tpp := ncu_traffic_per_point(method, kvar["variant"])) else None),
                         "peak_kind": peak_kind,
                         "kernel": f"{tma_kernel_name(kvar['variant'])} (persistent TMA fused stencil pass, FP32)",
                         "variant": kvar,
                         "avg_launch_us": avg_launch_ms * 1e3, "launches": kern_n,
                         "alg_bytes_per_launch": per_launch_bytes,
                         "timing": "CUDA events around every pass of one extra simulation after the timed region"},
            "cpu_baseline": {"value": cpu_tts, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": cpu_desc, "extrapolated": True},
            "e2e": {"value": e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
            "leapfrog_f32": (brief(lf) if lf else
                             ("no leap-frog step down to 1/32 of the stability step reaches the "
                              "target in FP32" if study else None)),
            "leapfrog_f64": brief(lf64) if lf64 else None,
            "best_per_method": {k_: {"m": c.m, "dt_over_leapfrog_step": round(c.dt / dt_cfl, 4),
                                     "time_to_solution_s": c.cost_s, "seismo_rel_err": c.err}
                                for k_, c in best_per_method.items()},
            "fp64_single_shot_s": (extras.get("fp64_single_shot") or {}).get("time_to_solution_s"),
            "fwi_gradient": ({k_: fp.get(k_) for k_ in ("method", "m", "dt_ms", "nsteps", "seconds",
                                                        "forward_s", "backward_s", "gradient_finite")}
                             if fp else None),
            "fwi_gradient_krylov": ({**{k_: fk.get(k_) for k_ in ("m", "dt_ms", "nsteps", "seconds",
                                                                  "forward_s", "backward_s", "stored_bytes",
                                                                  "adjoint")},
                                     "recomputing_s": (fk.get("recomputing_forward_arnoldi") or {}).get("seconds")}
                                    if fk else None),
            "config5_3d": ({"selected": {k_: (x3.get("selected") or {}).get(k_) for k_ in
                                         ("method", "m", "dt_over_leapfrog_step", "time_to_T_s",
                                          "seismo_rel_err_vs_fp64")},
                            "leapfrog_f32": {k_: (x3.get("leapfrog_best") or {}).get(k_) for k_ in
                                             ("dt_over_leapfrog_step", "time_to_T_s", "seismo_rel_err_vs_fp64")},
                            "roofline_frac": x3.get("roofline_frac"),
                            "pass_roofline_frac": {k_: v_.get("frac") for k_, v_ in
                                                   (x3.get("pass_rooflines") or {}).items()},
                            "pml": x3.get("pml")} if x3 else None),
            "config1_fp64": ({"selected": f1.get("selected"), "leapfrog": f1.get("leapfrog")}
                             if f1 else None),
            "bf16_storage": ([{"method": k_, "m": v[0], "dt_ms": v[1] * 1e3, "seismo_rel_err": v[2],
                               "seismo_rel_err_fp32": v[3]} for k_, v in study.bf16.items()]
                             if study else None),
            "search_s": study.seconds if study else None,
            "reference_self_check": study.ref_self_check if study else None,
            "run_s": time.perf_counter() - t_run,
        }
        line = json_line(result)
        if args.detail_out:
            detail = dict(result)
            detail.update(extras)
            detail["checked_problems"] = check
            detail["candidates"] = ([{"method": c.method, "m": c.m, "dt_ms": c.dt * 1e3,
                                      "seismo_rel_err": c.err, "growth": c.growth,
                                      "time_to_solution_s": c.cost_s} for c in study.candidates]
                                    if study else None)
            os.makedirs(os.path.dirname(os.path.abspath(args.detail_out)), exist_ok=True)
            with open(args.detail_out, "w") as f:
                f.write(json_line(detail) + "\n")
        print(line, flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def NOISE_LIMIT():
    from paper_2401_16322_gb300.tts import NOISE_GROWTH
    return NOISE_GROWTH


def main(argv=None):
    args = parse(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.case == "oracle":
        print(json_line({"oracle_full": oracle_full_runs(args.cpu_procs)}), flush=True)
        return 0
    if args.case == "cube":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json_line({"config5_3d": config5_3d(args.n3d, args.check3d)}), flush=True)
        return 0
    if args.case == "fwi":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json_line({"fwi_gradient": fwi_gradient_step(*DEFAULT_SELECTION),
                         "fwi_gradient_krylov": fwi_gradient_step("krylov", 20, 8.0)}), flush=True)
        return 0
    if args.case == "signal":
        import torch
        from paper_2401_16322_gb300 import single_signal
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        out = {"single_signal": single_signal.run(log=log)}
        if args.detail_out:
            with open(args.detail_out, "w") as f:
                f.write(json_line(out) + "\n")
        print(json_line(out), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""Time-to-solution search on the GPU (the paper's Delta-t_max criterion, Secs. 4.2 and 5.2).

For a workload (a list of velocity models with shots and surface receivers) this module

1. computes an FP64 reference seismogram for a few sampled problems with a high-accuracy
   setting of the same spatial discretisation (Faber, degree 30, at dt_ref = the leap-frog
   stability step, where the Faber coefficients beyond degree 30 are far below 1e-14; checked
   against dt_ref/2 by the reference self-check);
2. for every method and m, finds Delta-t_max: the largest step, an integer multiple k of the
   leap-frog step, whose FP32 seismograms on the sampled problems are within the target
   (1e-4 relative L2 over receivers x samples) of the reference at common sample times.  The
   multiples are scanned from the largest down and the scan stops at the first pass;
3. times one step of every (method, m) that has a Delta-t_max on the full batched workload;
4. selects the cheapest (steps x time per step).

Faber degree 20..120 is scanned up to 32 x the leap-frog step, Krylov dimension 10..40 up to
24 x (the paper's grid is 4..16 x), Krylov 20..40 with an orthogonalisation window of 2
("krylov-w2"), HORK 8..32 up to 12 x in its low-storage form and in Horner form
("hork-horner"); leap-frog itself, in FP32 (difference form) and in FP64, at
1 .. 1/32 of its step (largest passing step).
"""
import math
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .ewave import Batch, EwaveError, Model
from .workloads import Shot, Workload, t0_for

S2_MIN = {8: 6.501587301587302, 4: 16.0 / 3.0}   # |min symbol| of the centred 2nd derivative


def leapfrog_step(c_max, dx, order=8, dims=2):
    """Leap-frog stability step 2 / omega_max, omega_max = c_max sqrt(dims |S2|) / dx."""
    return 2.0 * dx / (c_max * math.sqrt(dims * S2_MIN[order]))


def pml_beta0(c_max, pml, dx, reflection=1e-3):
    """beta0 = 3 c_max / (2 delta) ln(1/R), R = 1e-3 (the model-parameter choice)."""
    return 3.0 * c_max / (2.0 * pml * dx) * math.log(1.0 / reflection)


@dataclass
class Candidate:
    method: str
    m: int
    dt: float
    err: float = float("nan")
    step_ms: float = float("nan")
    nsteps: int = 0
    growth: float = float("nan")     # white-noise norm growth over NOISE_STEPS steps

    @property
    def cost_s(self):
        return self.step_ms * self.nsteps * 1e-3

    def label(self):
        return f"{self.method}(m={self.m}, dt={self.dt * 1e3:.3f} ms)"


def build_models(workloads: List[Workload], precision, p=12, c_max=None, dx=None,
                 capacity=0, stream=None):
    """One Model per workload (all its shots), sources and receivers set, common beta0."""
    cm = c_max if c_max is not None else max(float(w.c.max()) for w in workloads)
    models = []
    for w in workloads:
        b0 = pml_beta0(cm, w.pml, w.dx)
        nrec = max(len(s.rec) for s in w.shots)
        md = Model(w.nx, w.ny, w.dx, w.order, w.pml, b0, w.free_surface, precision=precision,
                   nshots=len(w.shots), p=p, max_receivers=nrec, stream=stream)
        md.set_velocity(w.c)
        for k, s in enumerate(w.shots):
            md.set_source_receivers(k, s.sx, s.sy, w.f_peak, t0_for(w.f_peak), 1.0, s.rec)
        if capacity:
            md.bind_seismogram(capacity)
        models.append(md)
    return models


def common_ellipse(models, c_max):
    """Set one Faber ellipse (the widest of the models') on every model."""
    ells = [m.faber_ellipse() for m in models]
    best = max(ells, key=lambda e: e[0] * (1 - e[2]))
    for m in models:
        m.set_faber_ellipse(*best)
    return best


# local error tolerance of the adaptive Krylov candidate ("krylov-adaptive", m = m_max)
ADAPTIVE_TOL = 1e-6


def batch_step(batch, method, t, dt, m, nsteps):
    """Advance a batch; "krylov_adaptive" (the search's "krylov-adaptive") runs the adaptive
    Krylov step (m = m_max)."""
    if method == "krylov_adaptive":
        batch.step_krylov_adaptive(t, dt, ADAPTIVE_TOL, 1, m, nsteps)
    else:
        batch.step(method, t, dt, m, nsteps)


def base_method(models, method):
    """Map a candidate method name to the library's: "krylov-wQ" is Krylov with an
    orthogonalisation window of Q, "hork-horner" HORK evaluated in Horner form and
    "leapfrog-difference" leap-frog in difference form (set on every model; every other name
    resets them)."""
    from .ewave import LEAPFROG_AVERAGED, LEAPFROG_DIFFERENCE
    window = int(method[len("krylov-w"):]) if method.startswith("krylov-w") else 0
    for md in models:
        md.set_krylov_window(window)
        md.set_hork_form("horner" if method == "hork-horner" else "low-storage")
        if method.startswith("leapfrog"):
            md.set_leapfrog_variant(LEAPFROG_DIFFERENCE if method == "leapfrog-difference"
                                    else LEAPFROG_AVERAGED)
    if window:
        return "krylov"
    if method == "krylov-adaptive":
        return "krylov_adaptive"
    return {"hork-horner": "hork", "leapfrog-difference": "leapfrog"}.get(method, method)


def simulate(models, batch, method, m, dt, T, variant=0):
    """Run a fresh simulation to time T on every model; returns the number of steps."""
    method = base_method(models, method)
    nsteps = int(round(T / dt))
    for md in models:
        if md.capacity < nsteps:
            md.bind_seismogram(nsteps)
        md.reset_state()
        md.ensure_workspace(method, m)
    if method == "krylov_adaptive" and batch is None:
        for md in models:
            md.step_krylov_adaptive(0.0, dt, ADAPTIVE_TOL, 1, m, nsteps)
            md.sync()
        return nsteps
    if batch is None:
        for md in models:
            if method == "leapfrog":
                md.step_leapfrog(0.0, dt, nsteps, variant)
            else:
                md.step(method, 0.0, dt, m, nsteps)
            md.sync()
    else:
        batch_step(batch, method, 0.0, dt, m, nsteps)
        batch.sync()        # a non-finite result or a timed-out wait belongs to this run
    return nsteps


def sampled_workloads(workloads: List[Workload], picks):
    """Single-shot copies (model index, shot index) used for the error measurement."""
    out = []
    for wi, si in picks:
        w = workloads[wi]
        out.append(Workload(f"{w.name}-shot{si}", w.nx, w.ny, w.dx, w.order, w.pml,
                            w.free_surface, w.c, [w.shots[si]], w.f_peak, w.T))
    return out


def seismograms(models, nsteps):
    return [md.seismogram(0, len(w_rec), nsteps) for md, w_rec in models]


def rel_l2_common(seis, dt, ref, dt_ref):
    """Relative L2 error of ``seis`` (samples at (s+1) dt) against ``ref`` (at (s+1) dt_ref),
    over the sample times both contain (dt and dt_ref are integer multiples)."""
    if dt >= dt_ref:
        k = int(round(dt / dt_ref))
        n = min(seis.shape[0], ref.shape[0] // k)
        a, b = seis[:n], ref[k - 1::k][:n]
    else:
        k = int(round(dt_ref / dt))
        n = min(seis.shape[0] // k, ref.shape[0])
        a, b = seis[k - 1::k][:n], ref[:n]
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den)


@dataclass
class Study:
    dt_cfl: float
    dt_ref: float
    ref_method: str
    ref_m: int
    candidates: List[Candidate] = field(default_factory=list)
    selected: Optional[Candidate] = None
    leapfrog: Optional[Candidate] = None          # FP32 leap-frog (None: never reaches target)
    leapfrog_f64: Optional[Candidate] = None
    ref_self_check: float = float("nan")
    refs: list = field(default_factory=list)       # FP64 reference seismograms (sampled problems)
    ref_workloads: list = field(default_factory=list)
    bf16: dict = field(default_factory=dict)   # method -> (m, dt, error) with bfloat16 storage
    noise_problems: int = 0                    # problems (one shot per model) of the stability check
    seconds: float = 0.0


# (method, m values, step multiples k of the leap-frog step, scanned from the largest down)
SCAN_PLAN = (
    ("faber", (20, 25, 30, 35, 40, 45, 50, 55, 60, 70, 80, 100, 120), tuple(range(32, 1, -1))),
    ("krylov", (10, 15, 20, 30, 40), tuple(range(24, 1, -1))),
    ("krylov-w2", (20, 30, 40), tuple(range(24, 1, -1))),
    ("hork", (8, 12, 16, 20, 24, 28, 32), tuple(range(12, 0, -1))),
    ("hork-horner", (8, 12, 16, 20, 24, 28, 32), tuple(range(12, 0, -1))),
    ("krylov-adaptive", (40,), (24, 16, 12, 8, 6, 4, 3, 2)),
)
LEAPFROG_DIVISORS = (1, 2, 3, 4, 6, 8, 12, 16, 24, 32)
# Stability check of the polynomial integrators: a setting that meets the error target must
# also keep seeded white noise (every mode of the discrete operator excited, source off)
# from growing more than NOISE_GROWTH between step NOISE_STEPS and step 2 NOISE_STEPS on the
# sampled problems.  1.1 per 100 steps bounds the growth of any mode over a run of a few
# hundred steps to well under 2 x: a setting whose top eigenvalues lie outside the
# stability region fails it even when the smooth source barely excites them.
NOISE_STEPS = 100
NOISE_GROWTH = 1.1
POLYNOMIAL = ("faber", "hork", "hork-horner", "rk32", "rk44")


def dt_max_scan(ks, evaluate, target):
    """Delta-t_max search for one (method, m) (Secs. 4.2, 5.2): evaluate the candidates in
    the given order (largest step first) and stop at the first whose error meets the target.
    ``evaluate(k)`` returns the error (inf for a failed run).  Returns (k or None, [(k, err)])."""
    seen = []
    for k in ks:
        e = float(evaluate(k))
        seen.append((k, e))
        if e <= target:
            return k, seen
    return None, seen


def _eval_candidate(models, batch, refs, sw, c, T, dt_ref, log):
    try:
        c.nsteps = simulate(models, batch, c.method, c.m, c.dt, T)
        errs = [rel_l2_common(md.seismogram(0, len(w.shots[0].rec), c.nsteps), c.dt, r, dt_ref)
                for md, w, r in zip(models, sw, refs)]
        c.err = max(errs) if all(np.isfinite(errs)) else float("inf")
    except Exception as e:     # non-finite Arnoldi etc.: the candidate fails the target
        c.err = float("inf")
        log(f"  {c.label()}: {e}")
    return c.err


def noise_growth(models, batch, method, m, dt, t_quiet, nsteps=NOISE_STEPS, seed=97):
    """Stability of a setting on the actual spectrum of each discrete operator: from seeded
    white noise in u and v (source silent, t >= t_quiet) take ``nsteps`` steps, then
    ``nsteps`` more, and return the largest ||U_2N|| / ||U_N|| over the models.  Bounded
    dynamics give O(1) (the first segment absorbs the transfer between u and v and the PML's
    transients); a mode with |R| > 1 grows geometrically.  The smooth source of a shot
    barely excites the top of the spectrum, so the error scan alone cannot see it."""
    from .workloads import random_state
    method = base_method(models, method)
    for q, md in enumerate(models):
        md.ensure_workspace(method, m)
        md.reset_state()
        npts = md.nx * md.ny * (md.nz or 1)
        u, v = random_state([(npts,), (npts,)], seed + q)
        md.set_state(0, np.concatenate([u, v, np.zeros(md.n - 2 * npts)]))
    try:
        batch.step(method, t_quiet, dt, m, nsteps)
        batch.sync()
        mid = [float(np.linalg.norm(md.get_state(0))) for md in models]
        batch.step(method, t_quiet + nsteps * dt, dt, m, nsteps)
        batch.sync()
    except EwaveError as e:
        if "NONFINITE" in str(e):       # the noise grew past the floating-point range
            return float("inf")
        raise
    g = 0.0
    for md, a in zip(models, mid):
        b = float(np.linalg.norm(md.get_state(0)))
        g = max(g, b / a if np.isfinite(a) and np.isfinite(b) and a > 0 else float("inf"))
    return g


def _time_step(full_batch, full_models, method, m, dt, t_live):
    """ms per step of (method, m, dt) on the full workload, on a developed wavefield: from
    rest the Arnoldi process breaks down after p vectors (only the source tail spans the
    space), which would make Krylov steps look cheaper than they are."""
    import torch
    method = base_method(full_models, method)
    for md in full_models:
        md.ensure_workspace(method, m)
        md.reset_state()
    batch_step(full_batch, method, t_live - 2 * dt, dt, m, 2)   # inject the source, warm the graph
    full_batch.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ns = 2
    e0.record()
    batch_step(full_batch, method, t_live, dt, m, ns)
    e1.record()
    full_batch.sync()
    return e0.elapsed_time(e1) / ns


def run_study(workloads: List[Workload], picks, T, target=1e-4, plan=SCAN_PLAN,
              full_batch=None, full_models=None, full_models_f64=None, ref_m=30, p_ref=20,
              p=12, log=print, self_check=False, precision="f32"):
    """Delta-t_max search for every (method, m) of ``plan`` on the sampled problems, then the
    step time of each (method, m) on the full workload (``full_batch``/``full_models``; FP64
    leap-frog on ``full_models_f64`` when given).  Returns a Study."""
    t_start = time.time()
    c_max = max(float(w.c.max()) for w in workloads)
    dx = workloads[0].dx
    order = workloads[0].order
    dt_cfl = leapfrog_step(c_max, dx, order)
    dt_ref = dt_cfl
    sw = sampled_workloads(workloads, picks)
    # FP64 reference on the sampled problems, batched
    ref_models = build_models(sw, "f64", p=p_ref, c_max=c_max)
    ell = common_ellipse(ref_models, c_max)
    ref_batch = Batch(ref_models)
    n_ref = simulate(ref_models, ref_batch, "faber", ref_m, dt_ref, T)
    refs = [md.seismogram(0, len(w.shots[0].rec), n_ref) for md, w in zip(ref_models, sw)]
    st = Study(dt_cfl, dt_ref, "faber", ref_m, refs=refs, ref_workloads=sw)
    if self_check:
        n2 = simulate(ref_models, ref_batch, "faber", ref_m, dt_ref / 2, T)
        refs2 = [md.seismogram(0, len(w.shots[0].rec), n2) for md, w in zip(ref_models, sw)]
        st.ref_self_check = max(rel_l2_common(a, dt_ref, b, dt_ref / 2) for a, b in zip(refs, refs2))
        log(f"reference self-check (dt_ref vs dt_ref/2): {st.ref_self_check:.3e}")
    log(f"reference: FP64 faber m={ref_m} dt={dt_ref * 1e3:.3f} ms, {n_ref} steps "
        f"({time.time() - t_start:.1f} s)")
    t_quiet = T + 20.0 / workloads[0].f_peak + t0_for(workloads[0].f_peak)

    noise = {}            # models and batch of the stability check (set below)

    def scan(models, batch, method, m, ks, to_dt, out):
        def ev(k):
            c = Candidate(method, m, to_dt(k))
            out.append(c)
            err = _eval_candidate(models, batch, refs, sw, c, T, dt_ref, log)
            if err <= target and method in POLYNOMIAL:
                nm, nb = noise.get("models", models), noise.get("batch", batch)
                try:
                    c.growth = noise_growth(nm, nb, method, m, c.dt, t_quiet)
                except Exception as e:
                    c.growth = float("inf")
                    log(f"  {c.label()} noise test: {e}")
                if not c.growth <= NOISE_GROWTH:
                    log(f"  {c.label()}: error {err:.3e} but white noise grows {c.growth:.3g} x "
                        f"between steps {NOISE_STEPS} and {2 * NOISE_STEPS}: rejected")
                    c.err = float("inf")
            return c.err
        return dt_max_scan(ks, ev, target)[0]

    # FP64 leap-frog on the sampled problems (reuses the reference models)
    lf64 = []
    scan(ref_models, ref_batch, "leapfrog", 1, LEAPFROG_DIVISORS, lambda k: dt_cfl / k, lf64)
    ref_batch.close()
    for md in ref_models:
        md.close()
    # FP32 candidates on the sampled problems
    cand_models = build_models(sw, precision, p=p, c_max=c_max)
    for md in cand_models:
        md.set_faber_ellipse(*ell)
    cand_batch = Batch(cand_models)
    # the stability check runs on one shot of every model: the spectrum is the model's, and a
    # setting that is stable on the sampled problems can still have growing modes on another
    # model of the batch
    noise_models = build_models(sampled_workloads(workloads, [(q, 0) for q in range(len(workloads))]),
                                precision, p=p, c_max=c_max)
    for md in noise_models:
        md.set_faber_ellipse(*ell)
    noise_batch = Batch(noise_models)
    st.noise_problems = len(noise_models)
    noise["models"], noise["batch"] = noise_models, noise_batch
    cands, best_k = [], {}
    for method, ms, ks in plan:
        for m in ms:
            k = scan(cand_models, cand_batch, method, m, ks, lambda k: k * dt_cfl, cands)
            best_k[method, m] = k
            log(f"  {method} m={m}: dt_max = " + (f"{k} x leap-frog step" if k else "none in range")
                + f" ({time.time() - t_start:.1f} s)")
    # FP32 leap-frog in difference form (2D): the plain form's 2u^n - u^{n-1} puts an FP32
    # rounding error into the velocity every step, and its error stalls near 2e-4
    lf = []
    lf_name = "leapfrog-difference" if precision == "f32" else "leapfrog"
    scan(cand_models, cand_batch, lf_name, 1, LEAPFROG_DIVISORS, lambda k: dt_cfl / k, lf)
    # storage-precision experiment: for Faber and HORK, the passing FP32 (m, dt) with the
    # fewest passes per unit time, again on the sampled problems with every stored vector
    # rounded to bfloat16
    for method in ("faber", "hork", "hork-horner"):
        passing_s = [c for c in cands if c.err <= target and c.method == method and precision == "f32"]
        if not passing_s:
            continue
        best = min(passing_s, key=lambda c: c.m / c.dt)
        for md in cand_models:
            md.set_storage_rounding(True)
        probe = Candidate(best.method, best.m, best.dt)
        err = _eval_candidate(cand_models, cand_batch, refs, sw, probe, T, dt_ref, log)
        for md in cand_models:
            md.set_storage_rounding(False)
        st.bf16[method] = (best.m, best.dt, err, best.err)
        log(f"  bfloat16 storage, {probe.label()}: error {err:.3e} (FP32 {best.err:.3e})")
    cand_batch.close()
    for md in cand_models:
        md.close()
    noise_batch.close()
    for md in noise_models:
        md.close()
    # step time of every (method, m) with a passing step, on the full workload; the step
    # time does not depend on dt, so it applies to every passing candidate of that pair
    if full_batch is not None:
        t_live = t0_for(workloads[0].f_peak)
        step_ms = {}
        for (method, m), k in best_k.items():
            if k is None:
                continue
            try:
                step_ms[method, m] = _time_step(full_batch, full_models, method, m, k * dt_cfl, t_live)
            except EwaveError as e:
                # passed on the sampled problems but not on the whole batch: not a solution
                log(f"  {method} m={m} at {k} x leap-frog step fails on the full workload: {e}")
                for c in cands:
                    if (c.method, c.m) == (method, m) and c.err <= target:
                        c.err = float("inf")
        for c in cands:
            if c.err <= target and (c.method, c.m) in step_ms:
                c.step_ms = step_ms[c.method, c.m]
        lf_pass = [c for c in lf if c.err <= target]
        if lf_pass:
            lf_pass[0].step_ms = _time_step(full_batch, full_models, "leapfrog", 1, lf_pass[0].dt, t_live)
        lf64_pass = [c for c in lf64 if c.err <= target]
        if lf64_pass and full_models_f64 is not None:
            fb64 = Batch(full_models_f64)
            lf64_pass[0].step_ms = _time_step(fb64, full_models_f64, "leapfrog", 1, lf64_pass[0].dt, t_live)
            fb64.close()
    passing = [c for c in cands if c.err <= target and np.isfinite(c.step_ms)]
    st.candidates = cands + lf + lf64
    st.selected = min(passing, key=lambda c: c.cost_s) if passing else None
    lf_pass = [c for c in lf if c.err <= target and np.isfinite(c.step_ms)]
    st.leapfrog = lf_pass[0] if lf_pass else None
    lf64_pass = [c for c in lf64 if c.err <= target and np.isfinite(c.step_ms)]
    st.leapfrog_f64 = lf64_pass[0] if lf64_pass else None
    st.seconds = time.time() - t_start
    for c in st.candidates:
        log(f"  {c.label():34s} err {c.err:.3e}  step {c.step_ms:.3f} ms  steps {c.nsteps}  "
            f"cost {c.cost_s:.3f} s")
    return st

"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The whole batched workload (64 shots on 1001 x 501 plus eight models of 201 x 101 ..
801 x 401; 33.3 M grid points, FP32, one tile work list, persistent TMA passes, CUDA graphs)
is advanced by Faber steps of degree 50 at 8 x the leap-frog step.  Sampled problems start
from seeded smooth states; the oracle recomputes those problems independently.  The rest of
the batch starts from rest and is stepped in the same launches."""
import numpy as np
import pytest

from _helpers import TOL, flatten, rel_l2
from oracle.faber import faber_step
from oracle.model import Model as OModel
from oracle.model import unflatten
from oracle.operator import apply_H
from oracle.source import PointSource
from paper_2401_16322_gb300.workloads import config_batched, smooth_random_state, t0_for

pytestmark = pytest.mark.gpu

C_MAX = 4500.0
PICKS = [(0, 32), (1, 0), (5, 0)]          # (model, shot)


def _oracle_model(w):
    from paper_2401_16322_gb300.tts import pml_beta0
    return OModel(w.nx, w.ny, w.dx, w.order, w.pml, pml_beta0(C_MAX, w.pml, w.dx), w.free_surface, w.c)


def test_fullsize_batched_faber_steps_match_oracle_on_sampled_problems():
    import torch
    from paper_2401_16322_gb300 import Batch
    from paper_2401_16322_gb300.tts import build_models, common_ellipse, leapfrog_step
    wl = config_batched()
    models = build_models(wl, "f32", p=12, c_max=C_MAX)
    ell = common_ellipse(models, C_MAX)
    B = Batch(models)
    dt = 8 * leapfrog_step(C_MAX, wl[0].dx)
    deg, nsteps, t = 50, 2, t0_for(wl[0].f_peak) - 0.02
    init = {}
    for (wi, si) in PICKS:
        om = _oracle_model(wl[wi])
        U0 = tuple(smooth_random_state([f.shape for f in om.zeros_state()], 700 + wi * 100 + si))
        models[wi].set_state(si, flatten(U0))
        init[wi, si] = U0
    B.step("faber", t, dt, deg, nsteps)
    torch.cuda.synchronize()
    for (wi, si), U0 in init.items():
        w = wl[wi]
        om = _oracle_model(w)
        s = w.shots[si]
        src = PointSource(om, s.sx, s.sy, w.f_peak, t0_for(w.f_peak), 1.0, p=12)
        U = U0
        for n in range(nsteps):
            U = faber_step(om, U, src, t + n * dt, dt, deg, ell)
        got = models[wi].get_state(si)
        err = rel_l2(got, flatten(U))
        assert err < 3 * TOL["f32"], ((wi, si), err)


def test_fullsize_operator_matches_oracle():
    """H applied to a smooth field on the full 1001 x 501 grid (8th order, free surface)."""
    from paper_2401_16322_gb300.tts import build_models
    w = config_batched(nshots=1)[0]
    for prec, tol in (("f32", TOL["f32"]), ("f64", TOL["f64"])):
        md = build_models([w], prec, p=12, c_max=C_MAX)[0]
        om = _oracle_model(w)
        x = flatten(smooth_random_state([f.shape for f in om.zeros_state()], 55))
        ref = flatten(apply_H(om, unflatten(om, x)))
        assert rel_l2(md.apply(x), ref) < tol
        md.close()

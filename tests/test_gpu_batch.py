"""GPU batching: several models of uneven sizes (and several shots per model) stepped in the
same kernel launches give the same result as stepping them one at a time, and match the
oracle.  Covers the tile work list and the persistent TMA pass across problems."""
import numpy as np
import pytest

from _helpers import TOL, flatten, oracle_ellipse, oracle_model, rel_l2
from oracle.simulate import receiver_nodes, run
from oracle.source import PointSource
from paper_2401_16322_gb300.workloads import layered, smooth_random_state

pytestmark = pytest.mark.gpu

SIZES = [(83, 37), (130, 61), (45, 20)]


def _models(prec, nshots=2, p=8):
    from paper_2401_16322_gb300 import Model
    oms, gms, shots = [], [], []
    for q, (nx, ny) in enumerate(SIZES):
        om = oracle_model(nx, ny, layered(nx, ny, 10 + q), pml=8, fs=True)
        rec = np.array([[x * om.dx, 0.0] for x in range(2, nx - 2, 9)])
        g = Model(nx, ny, om.dx, 8, om.pml, om.beta0, True, precision=prec, nshots=nshots, p=p,
                  max_receivers=len(rec))
        g.set_velocity(om.c)
        sh = []
        for s in range(nshots):
            sx = (nx // 3 + s * (nx // 3)) * om.dx
            g.set_source_receivers(s, sx, 2 * om.dx, 20.0, 0.06, 1e3, rec)
            sh.append((sx, rec))
        oms.append(om)
        gms.append(g)
        shots.append(sh)
    return oms, gms, shots


def _init(oms, gms, nshots, at_rest=False):
    """Smooth random fields; ``at_rest``: displacement only (v = w = 0).  The Krylov step on
    a state whose v and w are O(1) beside an O(1) u is unphysical (v ~ omega u) and makes the
    Euclidean Arnoldi process amplify round-off ~500x on small PML-dominated grids; from rest
    the amplification is ~10x, so the FP64 1e-12 bar tests the kernels, not the conditioning."""
    U0 = {}
    for q, (om, g) in enumerate(zip(oms, gms)):
        for s in range(nshots):
            U = tuple(smooth_random_state([f.shape for f in om.zeros_state()], 100 + 10 * q + s))
            if at_rest:
                U = (U[0], 0 * U[1], 0 * U[2], 0 * U[3])
            U0[q, s] = U
            g.set_state(s, flatten(U))
    return U0


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("method,m", [("faber", 14), ("hork", 6), ("rk44", 0), ("krylov", 8)])
def test_batch_equals_oracle(prec, method, m):
    from paper_2401_16322_gb300 import Batch
    nshots, dt, t, nsteps = 2, 1.1e-3, 0.04, 2
    oms, gms, shots = _models(prec, nshots)
    ell = oracle_ellipse(oms[0])
    for g in gms:
        g.set_faber_ellipse(*ell)
        g.bind_seismogram(nsteps)
    U0 = _init(oms, gms, nshots, at_rest=(method == "krylov"))
    B = Batch(gms)
    B.step(method, t, dt, m, nsteps)
    for q, (om, g) in enumerate(zip(oms, gms)):
        for s in range(nshots):
            sx, rec = shots[q][s]
            src = PointSource(om, sx, 2 * om.dx, 20.0, 0.06, amp=1e3, p=8)
            U, S = run(om, method, dt, nsteps, src=src, rec_nodes=receiver_nodes(om, rec), m=m,
                       U0=U0[q, s], t0=t, faber_params=ell)
            tol = TOL[prec] * (3 if prec == "f32" else 1)
            assert rel_l2(g.get_state(s), flatten(U)) < tol, (q, s)
            assert rel_l2(g.seismogram(s, len(rec), nsteps), S) < tol, (q, s)


def test_batch_bitwise_equals_single_models():
    """The FP32 batch launch and per-model launches run identical arithmetic per problem."""
    from paper_2401_16322_gb300 import Batch
    nshots = 2
    oms, gms, _ = _models("f32", nshots)
    ell = oracle_ellipse(oms[0])
    for g in gms:
        g.set_faber_ellipse(*ell)
    U0 = _init(oms, gms, nshots)
    B = Batch(gms)
    B.set_kernel_variant(0)        # the pass variants agree to rounding, not bitwise
    for g in gms:
        g.set_kernel_variant(0)
    B.step("faber", 0.04, 1.1e-3, 20, 3)
    batched = [[g.get_state(s) for s in range(nshots)] for g in gms]
    for (q, s), U in U0.items():
        gms[q].set_state(s, flatten(U))
    for g in gms:
        g.step_faber(0.04, 1.1e-3, 20, 3)
    for q, g in enumerate(gms):
        for s in range(nshots):
            assert np.array_equal(batched[q][s], g.get_state(s))


@pytest.mark.parametrize("variant", list(range(15)))
def test_every_kernel_variant_matches_oracle(variant):
    """Each persistent-kernel variant the autotuner may pick (tile height 16, 8, 18 or 20;
    8 to 20 consumer warps; 3 to 5 stages; one or two columns per thread) gives the oracle's
    result on uneven batched grids."""
    from paper_2401_16322_gb300 import Batch
    nshots, dt, t, nsteps, m = 2, 1.1e-3, 0.04, 2, 14
    oms, gms, shots = _models("f32", nshots)
    ell = oracle_ellipse(oms[0])
    for g in gms:
        g.set_faber_ellipse(*ell)
        g.bind_seismogram(nsteps)
    U0 = _init(oms, gms, nshots)
    B = Batch(gms)
    B.set_kernel_variant(variant)
    B.step("faber", t, dt, m, nsteps)
    assert B.kernel_variant()["variant"] == variant
    for q, (om, g) in enumerate(zip(oms, gms)):
        for s in range(nshots):
            sx, rec = shots[q][s]
            src = PointSource(om, sx, 2 * om.dx, 20.0, 0.06, amp=1e3, p=8)
            U, S = run(om, "faber", dt, nsteps, src=src, rec_nodes=receiver_nodes(om, rec), m=m,
                       U0=U0[q, s], t0=t, faber_params=ell)
            assert rel_l2(g.get_state(s), flatten(U)) < 3 * TOL["f32"], (variant, q, s)


def test_autotuner_picks_a_timed_variant():
    from paper_2401_16322_gb300 import Batch
    oms, gms, _ = _models("f32", 1)
    for g in gms:
        g.set_faber_ellipse(*oracle_ellipse(oms[0]))
    B = Batch(gms)
    B.step("faber", 0.04, 1.1e-3, 8, 1)
    info = B.kernel_variant()
    times = info["probe_us"]
    assert len(times) == 15 and 0 <= info["variant"] < len(times)
    assert all(t > 0 for t in times)
    assert times[info["variant"]] == min(times)


def test_bf16_storage_rounding_stores_bf16_values():
    """Storage-precision experiment: after HORK steps with bfloat16 storage rounding every
    stored value has a zero low half (exactly representable in bfloat16), and the result
    stays within the bfloat16 error bound of the FP32 run."""
    from paper_2401_16322_gb300.ewave import EwaveError
    oms, gms, _ = _models("f32", 1)
    om, g = oms[0], gms[0]
    U0 = smooth_random_state([f.shape for f in om.zeros_state()], 31)
    out = []
    for bf16 in (False, True):
        g.set_storage_rounding(bf16)
        g.set_state(0, flatten(U0))
        g.step("hork", 0.04, 1.0e-3, 8, 3)
        out.append(g.get_state(0))
    bits = out[1].astype(np.float32).view(np.uint32)
    assert np.all((bits & 0xFFFF) == 0)
    # 24 rounded passes, unit round-off 2^-8 each: a linear bound
    assert 1e-5 < rel_l2(out[1], out[0]) < 24 * 2.0 ** -8
    from paper_2401_16322_gb300 import Model
    m64 = Model(om.nx, om.ny, om.dx, om.order, om.pml, om.beta0, om.free_surface, precision="f64")
    with pytest.raises(EwaveError, match="UNSUPPORTED"):
        m64.set_storage_rounding(True)
    m64.close()


def test_white_noise_stability_check():
    """The search's stability check: from seeded white noise with the source silent, a HORK
    setting far outside its stability region grows, while a Faber setting whose ellipse
    encloses the spectrum does not (the PML only removes energy)."""
    from paper_2401_16322_gb300 import Batch
    from paper_2401_16322_gb300.tts import leapfrog_step, noise_growth
    oms, gms, _ = _models("f32", 1)
    for g, om in zip(gms, oms):
        g.set_faber_ellipse(*oracle_ellipse(om))
    B = Batch(gms)
    dt = 3.0 * leapfrog_step(float(max(om.c_max for om in oms)), oms[0].dx)
    grow_hork = noise_growth(gms, B, "hork", 6, dt, t_quiet=5.0, nsteps=60)
    grow_faber = noise_growth(gms, B, "faber", 40, dt, t_quiet=5.0, nsteps=60)
    assert grow_hork > 10.0
    assert grow_faber <= 2.0


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("variant", ["averaged", "difference"])
def test_batch_leapfrog_equals_oracle(prec, variant):
    """Leap-frog over uneven batched models (FP32: the persistent TMA step), an odd number of
    steps so that the final buffer swap runs; u and the w fields against the oracle."""
    from paper_2401_16322_gb300 import Batch
    from paper_2401_16322_gb300.ewave import LEAPFROG_AVERAGED, LEAPFROG_DIFFERENCE
    nshots, dt, t, nsteps = 2, 3e-4, 0.04, 5
    oms, gms, shots = _models(prec, nshots)
    for g in gms:
        g.bind_seismogram(nsteps)
        g.set_leapfrog_variant(LEAPFROG_DIFFERENCE if variant == "difference" else LEAPFROG_AVERAGED)
    U0 = _init(oms, gms, nshots, at_rest=True)
    B = Batch(gms)
    B.step("leapfrog", t, dt, 0, nsteps)
    for q, (om, g) in enumerate(zip(oms, gms)):
        n_u = om.nx * om.ny
        keep = np.ones(om.n, bool)
        keep[n_u:2 * n_u] = False                  # v is not advanced by leap-frog
        for s in range(nshots):
            sx, rec = shots[q][s]
            src = PointSource(om, sx, 2 * om.dx, 20.0, 0.06, amp=1e3, p=8)
            U, S = run(om, "leapfrog", dt, nsteps, src=src, rec_nodes=receiver_nodes(om, rec),
                       U0=U0[q, s], t0=t, lf_variant="averaged")
            tol = TOL[prec] * (3 if prec == "f32" else 1)
            assert rel_l2(g.get_state(s)[keep], flatten(U)[keep]) < tol, (q, s)
            assert rel_l2(g.seismogram(s, len(rec), nsteps), S) < tol, (q, s)

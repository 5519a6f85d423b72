"""GPU parity of every time integrator (Sec. 3) against the oracle, through the C ABI:
Faber, Krylov, HORK (augmented source, Eq. matrix_ampli), RK3-2, RK4-4 and leap-frog,
in FP64 (1e-12) and FP32 (1e-5 per step), with the source active and receivers recorded."""
import numpy as np
import pytest

from _helpers import TOL, flatten, gpu_model, oracle_ellipse, oracle_model, rel_l2
from oracle import faber, krylov, leapfrog, rk
from oracle.simulate import receiver_nodes, run
from oracle.source import PointSource
from paper_2401_16322_gb300.workloads import layered, smooth_random_state

pytestmark = pytest.mark.gpu

NX, NY = 83, 37          # 2 x 3 tiles, ragged in both directions


def _setup(prec, fs=True, order=8, p=10, seed=4):
    c = layered(NX, NY, seed)
    om = oracle_model(NX, NY, c, order=order, pml=10, fs=fs)
    rec = np.array([[x * om.dx, 0.0 if fs else 5 * om.dx] for x in range(3, NX - 3, 7)])
    g = gpu_model(om, prec, p=p, max_receivers=len(rec))
    sx, sy = 41 * om.dx + 3.0, (2 if fs else 18) * om.dx
    src = PointSource(om, sx, sy, 25.0, 0.05, amp=1e3, p=p)
    si, ri = g.set_source_receivers(0, sx, sy, 25.0, 0.05, 1e3, rec)
    assert (si[1], si[0]) == (src.j, src.i)
    rn = receiver_nodes(om, rec)
    assert np.array_equal(ri[:, ::-1], rn)          # integer indices: bit-exact
    U0 = tuple(smooth_random_state([f.shape for f in om.zeros_state()], 9))
    return om, g, src, rec, rn, U0


def _gpu_run(g, U0, method, t, dt, m, nsteps, capacity):
    g.bind_seismogram(capacity)
    g.set_state(0, flatten(U0))
    info = g.step(method, t, dt, m, nsteps)
    return g.get_state(0), info


CASES = [("faber", 12), ("faber", 30), ("krylov", 8), ("krylov", 16), ("hork", 1), ("hork", 2),
         ("hork", 7), ("rk32", 0), ("rk44", 0), ("faber", 1), ("faber", 2), ("krylov", 1)]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("method,m", CASES)
def test_integrator_matches_oracle(prec, method, m):
    om, g, src, rec, rn, U0 = _setup(prec)
    if method == "krylov":
        # displacement at rest: see tests/test_gpu_batch.py::_init on the conditioning
        U0 = (U0[0], 0 * U0[1], 0 * U0[2], 0 * U0[3])
    dt, t, nsteps = 1.2e-3, 0.03, 3
    if method == "faber":
        g.set_faber_ellipse(*oracle_ellipse(om))
    gs, _ = _gpu_run(g, U0, method, t, dt, m, nsteps, nsteps)
    U, S = run(om, method, dt, nsteps, src=src, rec_nodes=rn, m=m, U0=U0, t0=t)
    err = rel_l2(gs, flatten(U))
    assert err < TOL[prec] * (3 if prec == "f32" else 1), (method, m, err)
    Sg = g.seismogram(0, len(rec), nsteps)
    assert rel_l2(Sg, S) < (TOL[prec] * 3 if prec == "f32" else TOL[prec])


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("variant", ["averaged", "literal", "difference"])
def test_leapfrog_matches_oracle(prec, variant):
    """Both damping readings, and the averaged one in difference form (the same scheme in
    exact arithmetic: the oracle's averaged leap-frog is its reference)."""
    from paper_2401_16322_gb300.ewave import LEAPFROG_AVERAGED, LEAPFROG_DIFFERENCE, LEAPFROG_LITERAL
    code = {"averaged": LEAPFROG_AVERAGED, "literal": LEAPFROG_LITERAL,
            "difference": LEAPFROG_DIFFERENCE}[variant]
    ovar = "literal" if variant == "literal" else "averaged"
    om, g, src, rec, rn, U0 = _setup(prec)
    U0 = (U0[0], np.zeros_like(U0[1]), U0[2], U0[3])
    dt, t, nsteps = 4e-4, 0.03, 7                    # odd: exercises the final buffer swap
    g.bind_seismogram(nsteps)
    g.set_state(0, flatten(U0))
    g.step_leapfrog(t, dt, nsteps, code)
    gs = g.get_state(0)
    U, S = run(om, "leapfrog", dt, nsteps, src=src, rec_nodes=rn, U0=U0, t0=t, lf_variant=ovar)
    n_u = om.nx * om.ny
    ref = flatten(U)
    mask = np.ones(om.n, bool)
    mask[n_u:2 * n_u] = False                        # v is not advanced by leap-frog
    assert rel_l2(gs[mask], ref[mask]) < TOL[prec] * (3 if prec == "f32" else 1)
    assert rel_l2(g.seismogram(0, len(rec), nsteps), S) < TOL[prec] * (3 if prec == "f32" else 1)
    # continuing from the restored buffers gives the same as one longer call
    g.step_leapfrog(t + nsteps * dt, dt, 2, code)
    U2, _ = run(om, "leapfrog", dt, nsteps + 2, src=src, rec_nodes=rn, U0=U0, t0=t, lf_variant=ovar)
    assert rel_l2(g.get_state(0)[mask], flatten(U2)[mask]) < TOL[prec] * (3 if prec == "f32" else 1)


@pytest.mark.parametrize("order,fs", [(4, False), (8, False)])
def test_faber_and_krylov_without_free_surface(order, fs):
    om, g, src, rec, rn, U0 = _setup("f64", fs=fs, order=order)
    g.set_faber_ellipse(*oracle_ellipse(om))
    for method, m in (("faber", 20), ("krylov", 12)):
        if method == "krylov":
            U0 = (U0[0], 0 * U0[1], 0 * U0[2], 0 * U0[3])
        gs, _ = _gpu_run(g, U0, method, 0.02, 1.5e-3, m, 2, 2)
        U, _ = run(om, method, 1.5e-3, 2, src=src, rec_nodes=rn, m=m, U0=U0, t0=0.02)
        assert rel_l2(gs, flatten(U)) < TOL["f64"], method


def test_default_faber_ellipse_matches_oracle_reading():
    om, g, *_ = _setup("f64")
    ge = g.faber_ellipse()
    oe = oracle_ellipse(om)
    assert np.allclose(ge, oe, rtol=1e-12, atol=0)


def test_krylov_breakdown_reports_dimension():
    """A zero state with no source: |x| = |e_p| and the augmented tail space is only
    p-dimensional under J, so Arnoldi breaks down early (happy breakdown)."""
    nx, ny = 20, 18
    om = oracle_model(nx, ny, layered(nx, ny, 2), pml=4, fs=True)
    g = gpu_model(om, "f64", p=3)
    g.set_state(0, np.zeros(om.n))
    info = g.step_krylov(0.0, 1e-3, 10, 1)
    assert info == 3
    assert np.all(g.get_state(0) == 0.0)


def test_seismogram_indices_bit_exact():
    nx, ny = 50, 30
    om = oracle_model(nx, ny, layered(nx, ny, 2), pml=4, fs=True)
    g = gpu_model(om, "f32", max_receivers=6)
    rec = np.array([[0.0, 0.0], [14.999, 4.999], [15.0, 5.0], [490.0, 290.0], [104.9, 0.0], [255.0, 35.0]])
    si, ri = g.set_source_receivers(0, 245.0, 15.0, 10.0, 0.27, 1.0, rec)
    ref = receiver_nodes(om, rec)
    assert np.array_equal(ri[:, ::-1], ref)
    assert list(si) == [int(np.floor(245.0 / 10 + 0.5)), int(np.floor(15.0 / 10 + 0.5))]
    with pytest.raises(Exception):
        g.set_source_receivers(0, -6.0, 15.0, 10.0, 0.27, 1.0, rec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("m,q", [(12, 2), (16, 3)])
def test_krylov_with_orthogonalisation_window_matches_oracle(prec, m, q):
    """Incomplete orthogonalisation (window q): the GPU step equals the oracle's windowed
    Arnoldi step, with the source active."""
    om, g, src, rec, rn, U0 = _setup(prec)
    U0 = (U0[0], 0 * U0[1], 0 * U0[2], 0 * U0[3])
    dt, t, nsteps = 1.2e-3, 0.03, 3
    g.set_krylov_window(q)
    gs, _ = _gpu_run(g, U0, "krylov", t, dt, m, nsteps, nsteps)
    U = U0
    for n in range(nsteps):
        U = krylov.krylov_step(om, U, src, t + n * dt, dt, m, window=q)
    err = rel_l2(gs, flatten(U))
    assert err < TOL[prec] * (3 if prec == "f32" else 1), (m, q, err)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("form", ["low-storage", "horner"])
@pytest.mark.parametrize("m,k", [(1, 0.3), (2, 0.5), (7, 1.0), (24, 5.0)])
def test_hork_forms_match_oracle(prec, form, m, k):
    """Both evaluation orders of HORK(m) (the paper's low-storage stages with lambda_i;
    Horner: V_j = V_0 + (dt/j) H~ V_{j+1}) equal the oracle's HORK step, with the source
    active, up to k times the leap-frog step (m = 24 at 5x: the setting the step search
    selects).

    FP32 Horner bound: rounding made in pass j reaches the result multiplied by
    (dt lambda)^(j-1)/(j-1)!, and |dt lambda| <= 2k on this spectrum (the top of the interior
    spectrum is 2 / leap-frog step), so per step the error is at most about
    2^-24 max_j (2k)^j / j!; the tolerance is the larger of that over the steps and the usual
    FP32 one.  At k = 5 that is 5e-4 (measured 6.6e-5; the low-storage form 1.2e-6)."""
    import math
    from paper_2401_16322_gb300.tts import leapfrog_step
    om, g, src, rec, rn, U0 = _setup(prec)
    g.set_hork_form(form)
    dt = k * leapfrog_step(om.c_max, om.dx)
    t, nsteps = 0.03, 3
    gs, _ = _gpu_run(g, U0, "hork", t, dt, m, nsteps, nsteps)
    U, S = run(om, "hork", dt, nsteps, src=src, rec_nodes=rn, m=m, U0=U0, t0=t)
    tol = TOL[prec] * (3 if prec == "f32" else 1)
    if prec == "f32" and form == "horner":
        gain = max((2 * k) ** j / math.factorial(j) for j in range(m + 1))
        tol = max(tol, nsteps * 2.0 ** -24 * gain)
    err = rel_l2(gs, flatten(U))
    assert err < tol, (form, m, err, tol)
    assert rel_l2(g.seismogram(0, len(rec), nsteps), S) < tol


def test_hork_horner_and_low_storage_agree_fp64():
    om, g, src, rec, rn, U0 = _setup("f64")
    out = []
    for form in ("low-storage", "horner", "low-storage"):
        g.set_hork_form(form)
        out.append(_gpu_run(g, U0, "hork", 0.03, 4e-3, 16, 4, 4)[0])
    assert np.array_equal(out[0], out[2])           # switching back restores the same graph
    assert rel_l2(out[1], out[0]) < 1e-13


def test_leapfrog_difference_form_cuts_fp32_rounding():
    """Many small FP32 steps (1/12 of the stability step): the difference form stays much
    closer to the FP64 run than the plain form, whose 2u^n - u^{n-1} turns each step's
    rounding into a velocity error."""
    from paper_2401_16322_gb300.ewave import LEAPFROG_AVERAGED, LEAPFROG_DIFFERENCE
    from paper_2401_16322_gb300.tts import leapfrog_step
    errs = {}
    for variant in (LEAPFROG_AVERAGED, LEAPFROG_DIFFERENCE):
        out = {}
        for prec in ("f64", "f32"):
            om, g, src, rec, rn, U0 = _setup(prec)
            dt = leapfrog_step(om.c_max, om.dx) / 12
            nsteps = 600
            g.bind_seismogram(nsteps)
            g.set_state(0, flatten(tuple(0 * f for f in U0)))
            g.step_leapfrog(0.0, dt, nsteps, variant)
            out[prec] = g.seismogram(0, len(rec), nsteps)
            g.close()
        errs[variant] = rel_l2(out["f32"], out["f64"])
    assert errs[LEAPFROG_DIFFERENCE] < 0.5 * errs[LEAPFROG_AVERAGED], errs

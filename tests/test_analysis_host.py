"""Pins of the dispersion / dissipation analysis (host logic, no GPU): each amplification
factor against an independent route (direct iteration of the scheme on one eigenmode, the
Taylor remainder bound, the exact exponential)."""
import math

import numpy as np
import pytest

from paper_2401_16322_gb300.analysis import amplification, dispersion_dissipation


def test_leapfrog_root_matches_direct_iteration():
    dt = 1.0
    for theta in (0.1, 0.7, 1.5, 1.9):
        # u^{n+1} = 2 u^n - u^{n-1} - theta^2 u^n started on the mode zeta: the ratio is zeta
        z = amplification("leapfrog", 1, theta, dt)
        u_prev, u = 1.0 + 0j, complex(z)
        for _ in range(50):
            u_prev, u = u, 2 * u - u_prev - theta ** 2 * u
        assert abs(u / u_prev - z) < 1e-9
        assert abs(abs(z) - 1.0) < 1e-12                        # neutral for theta <= 2
        assert abs(np.angle(z) - math.acos(1 - theta ** 2 / 2)) < 1e-12
    assert abs(amplification("leapfrog", 1, 2.5, dt)) > 1.0     # unstable beyond 2


def test_rk32_matches_its_stages_on_one_mode():
    w, dt = 3.0, 0.2
    f = lambda y: 1j * w * y                                   # noqa: E731
    k1 = f(1.0)
    k2 = f(1.0 + dt / 2 * k1)
    k3 = f(1.0 + dt / 2 * k2)
    assert abs((1.0 + dt * k3) - amplification("rk32", 0, w, dt)) < 1e-14


def test_hork_within_the_taylor_remainder():
    for m in (4, 8, 16):
        for theta in (0.1, 0.5, 1.0):
            R = amplification("hork", m, theta, 1.0)
            bound = theta ** (m + 1) / math.factorial(m + 1)
            assert abs(R - np.exp(1j * theta)) <= 1.01 * bound + 1e-15


def test_faber_converges_to_the_exponential_inside_the_ellipse():
    ell = (2.0, -0.1, -0.8)          # ellipse: imaginary semi-axis gamma (1 - c1) = 3.6
    for theta in (0.5, 2.0, 3.0):
        R = amplification("faber", 60, theta, 1.0, ell)
        assert abs(R - np.exp(1j * theta)) < 1e-12
    d, p = dispersion_dissipation("faber", 60, 1.0, 3.0, ell)
    assert d < 1e-12 and p < 1e-12


def test_rk44_dissipates_and_lags():
    d, p = dispersion_dissipation("rk44", 0, 0.5, 2.0)        # omega dt up to 1
    assert 1e-4 < d < 2e-2 and 1e-5 < p < 1e-2


def test_hork_stability_edge_on_a_dense_spectrum():
    """The white-noise check of the step search rejects HORK settings whose amplification
    exceeds the exact propagator's on the discrete spectrum.  On the dense spectrum of a small
    layered PML model (oracle operator, FP64), R is evaluated at z = lambda dt for every
    eigenvalue lambda, damping included.  The operator has one real eigenvalue above zero
    (~0.07 1/s: a slow, non-oscillating mode of the damped operator, absent without damping),
    which the exact exponential grows too.  HORK 16 grows nothing faster than that at 2x and
    3x the leap-frog step and amplifies by ~2 at 4x: its Taylor polynomial leaves the unit
    disk near omega dt = 6 on the imaginary axis, and the top of the spectrum approaches
    2 / leap-frog step."""
    from oracle.model import Model, default_beta0
    from oracle.operator import assemble_H
    from paper_2401_16322_gb300.tts import leapfrog_step
    from paper_2401_16322_gb300.workloads import layered
    c = layered(30, 22, 5, vmin=1500, vmax=4500)
    m = Model(30, 22, 10.0, 8, 5, default_beta0(float(c.max()), 5, 10.0), True, c)
    ev = np.linalg.eigvals(assemble_H(m).toarray())
    dt_lf = leapfrog_step(float(c.max()), 10.0)
    top = np.abs(ev.imag).max() * dt_lf
    assert 1.8 < top < 2.0
    assert int((ev.real > 1e-6).sum()) == 1 and 0.0 < ev.real.max() < 0.2
    m0 = Model(30, 22, 10.0, 8, 5, 0.0, True, c)
    assert np.linalg.eigvals(assemble_H(m0).toarray()).real.max() < 1e-9
    for k, bound in ((2, None), (3, None), (4, 1.3)):
        grow = np.abs(amplification("hork", 16, ev / 1j, k * dt_lf)).max()
        exact = math.exp(ev.real.max() * k * dt_lf)
        if bound is None:
            assert grow <= exact * (1 + 1e-9), (k, grow, exact)
        else:
            assert grow > bound, (k, grow)


# ---------------------------------------------------------------- Sec. 4.1 trace measure
def _tone(n, k0, amp=1.0):
    return amp * np.cos(2 * np.pi * k0 * np.arange(n) / n)


def test_trace_errors_of_identical_traces_vanish():
    from paper_2401_16322_gb300.analysis import trace_errors
    t = np.arange(3118) * 0.417e-3
    a = (math.pi * 15.0) ** 2
    ricker = (1 - 2 * a * (t - 0.18) ** 2) * np.exp(-a * (t - 0.18) ** 2)
    assert max(trace_errors(ricker, ricker)) < 1e-14


def test_trace_errors_of_a_scaled_trace_are_its_log_amplitude():
    """F_ref = exp(k) F_appr with appr = 0.9 ref: k = ln(1/0.9) at every bin, l = 0."""
    from paper_2401_16322_gb300.analysis import trace_errors
    t = np.arange(3118) * 0.417e-3
    a = (math.pi * 15.0) ** 2
    ricker = (1 - 2 * a * (t - 0.18) ** 2) * np.exp(-a * (t - 0.18) ** 2)
    diss, disp = trace_errors(ricker, 0.9 * ricker)
    assert abs(diss - math.log(1 / 0.9)) < 1e-12 and disp < 1e-12


@pytest.mark.parametrize("k0,s", [(37, 1), (37, 5), (200, 2)])
def test_trace_errors_of_a_delayed_tone_are_its_phase_shift(k0, s):
    """A pure tone in bin k0 delayed by s samples: l = 2 pi k0 s / N, k = 0."""
    from paper_2401_16322_gb300.analysis import trace_errors
    n = 2048
    ref = _tone(n, k0)
    diss, disp = trace_errors(ref, np.roll(ref, s))
    assert diss < 1e-12 and abs(disp - 2 * np.pi * k0 * s / n) < 1e-12


def test_trace_errors_select_bins_above_one_percent_of_either_trace():
    """A spurious tone in the approximate trace counts once it passes 1 % of the reference
    peak (the union of the two amplitude tests), not below."""
    from paper_2401_16322_gb300.analysis import trace_errors
    n = 2048
    ref = _tone(n, 37)
    assert max(trace_errors(ref, ref + _tone(n, 300, 0.005))) < 1e-14
    diss, _ = trace_errors(ref, ref + _tone(n, 300, 0.02))
    assert diss > 1.0


def test_trace_errors_show_leapfrog_second_order():
    """On traces of the oracle (homogeneous 1.2 x 1 km at 10 m, c = 3 km/s, 15 Hz Ricker, one
    receiver 300 m from the source, T = 0.3 s, before any boundary reflection arrives), the
    leap-frog scheme's dispersion and dissipation errors against an HORK 8 reference at 1 ms
    (whose own errors by this measure against Faber 40 at 1 ms are ~1e-10) fall by 4 when dt
    halves: second order."""
    from oracle.model import Model
    from oracle.simulate import receiver_nodes, run
    from oracle.source import PointSource
    from paper_2401_16322_gb300.analysis import trace_errors
    m = Model(121, 101, 10.0, 8, 0, 0.0, False, np.full((101, 121), 3000.0))
    src = PointSource(m, 600.0, 700.0, 15.0, 0.08, amp=1e3, p=12)
    rec = receiver_nodes(m, np.array([[600.0, 400.0]]))
    _, ref = run(m, "hork", 1e-3, 300, src, rec, m=8)
    errs = []
    for dt in (1e-3, 0.5e-3, 0.25e-3):
        stride = int(round(1e-3 / dt))
        _, s = run(m, "leapfrog", dt, 300 * stride, src, rec)
        errs.append(trace_errors(ref[:, 0], s[stride - 1::stride, 0]))
    assert 0.01 < errs[0][1] < 0.03
    for a, b in zip(errs, errs[1:]):
        assert 3.6 < a[0] / b[0] < 4.4 and 3.6 < a[1] / b[1] < 4.4, errs

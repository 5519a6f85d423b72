"""Pins of the dispersion / dissipation analysis (host logic, no GPU): each amplification
factor against an independent route (direct iteration of the scheme on one eigenmode, the
Taylor remainder bound, the exact exponential)."""
import math

import numpy as np

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
    exceeds 1 on the discrete spectrum.  On the dense spectrum of a small layered PML model
    (oracle operator, FP64) HORK 16 is stable at 2x the leap-frog step, marginal at 3x and
    unstable at 4x: its Taylor polynomial leaves the unit disk near omega dt = 6 on the
    imaginary axis, and the top of the spectrum approaches 2 / leap-frog step."""
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
    grow = [np.abs(amplification("hork", 16, ev / 1j, k * dt_lf)).max() for k in (2, 3, 4)]
    assert grow[0] < 1.001 and grow[1] < 1.05 and grow[2] > 1.3

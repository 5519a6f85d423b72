"""Physics pin of the oracle: the 2D homogeneous-medium Green's function.

For u_tt = c^2 (u_xx + u_yy) + delta(x) r(t) (Eq. 1 without damping near the source, with
f = r(t)/dx^2 at a node standing in for the delta), u(R, t) = int G(R, s) r(t - s) ds with
G = H(ct - R) / (2 pi c sqrt(c^2 t^2 - R^2)).  With s = (R/c) cosh(phi) the singularity
goes away: u = 1/(2 pi c^2) int_0^{acosh(ct/R)} r(t - (R/c) cosh phi) d phi.
"""
import math

import numpy as np

from oracle.model import Model, default_beta0
from oracle.simulate import receiver_nodes, rel_l2, run
from oracle.source import PointSource, ricker


def _analytic(R, t, c, f, t0, nq=300):
    if c * t <= R:
        return 0.0
    Phi = math.acosh(c * t / R)
    x, w = np.polynomial.legendre.leggauss(nq)
    ph = 0.5 * Phi * (x + 1.0)
    vals = np.array([ricker(t - (R / c) * math.cosh(p), f, t0) for p in ph])
    return 0.5 * Phi * float(np.dot(w, vals)) / (2.0 * math.pi * c * c)


def test_greens_function_receivers():
    N, dx, c, f, t0 = 101, 10.0, 2000.0, 10.0, 0.2
    m = Model(N, N, dx, 8, 20, default_beta0(c, 20, dx), False, np.full((N, N), c))
    ctr = (N // 2) * dx
    src = PointSource(m, ctr, ctr, f, t0, p=12)
    rec = np.array([[ctr + 200.0, ctr], [ctr, ctr + 250.0], [ctr + 150.0, ctr + 150.0]])
    dt, T = 2e-3, 0.36
    ns = int(round(T / dt))
    _, S = run(m, "faber", dt, ns, src=src, rec_nodes=receiver_nodes(m, rec), m=24)
    ts = (np.arange(ns) + 1) * dt
    A = np.array([[_analytic(math.hypot(*(r - [ctr, ctr])), t, c, f, t0) for r in rec]
                  for t in ts])
    # measured 6.7e-6 at dx = 10 m (7.9e-8 at dx = 5 m): the discretisation error
    assert rel_l2(S, A) < 2e-5

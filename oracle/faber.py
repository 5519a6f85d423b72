"""Faber-polynomial exponential integrator (Sec. 3.2, "Faber approximation") of the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Recurrence (Sec. 3.2): F_0 = I, F_1 = H/gamma - c0 I, F_2 = F_1^2 - 2 c1 I,
F_j = F_1 F_{j-1} - c1 F_{j-2}; u^{n+1} = sum_{j=0}^m a_j F_j(H~) [u^n; e_p].

Readings (the paper defers gamma, c0, c1 and a_j to its earlier Faber paper):

* The recurrence is the Faber sequence of the exterior conformal map
  psi(w) = gamma (w + c0 + c1/w), which maps |w| = 1 onto an ellipse with centre gamma c0
  and semi-axes gamma (1 + c1) (real) and gamma (1 - c1) (imaginary); indeed
  F_j(psi(w)) = w^j + c1^j w^-j.  So gamma = (a_r + a_i)/2, c0 = centre/gamma and
  c1 = (a_r - a_i)/(a_r + a_i).
* Ellipse: the smallest axis-aligned ellipse through the corners of the rectangle
  [-beta_sum, 0] x [-omega, omega] with the same aspect (semi-axes sqrt(2) times the
  half-sides), centred at -beta_sum/2, where beta_sum = dims * beta0 and
  omega = kappa c_max sqrt(dims |S2|)/dx, S2 the minimum of the centred second-derivative
  symbol; kappa = 1.05 without and 1.30 with the free surface (its one-sided rows widen
  the imaginary extent of the spectrum by about 22 % on small grids).
* a_j are the Faber coefficients of z -> exp(dt z): the w^j coefficient of
  exp(dt psi(w)) on |w| = 1, computed by the trapezoid rule on N >= max(4m, 64) nodes.

Pins: tests/test_oracle_integrators.py (Bessel J/I closed forms, the Taylor special case, and
convergence of the step to the dense matrix exponential).
"""
import math

import numpy as np

from . import stencils as S
from .operator import apply_H
from .source import tail_apply


def symbol_min(order):
    """Minimum over theta of the centred second-derivative symbol d0 + 2 sum d_k cos(k theta)."""
    d = S.as_float(S.CENT[order])
    th = np.linspace(0.0, math.pi, 20001)
    sym = d[0] + 2.0 * sum(d[k] * np.cos(k * th) for k in range(1, len(d)))
    return float(sym.min())


def ellipse_params(c_max, beta0, dx, order, dims=2, free_surface=False):
    """(gamma, c0, c1) of the enclosing ellipse described in the module header."""
    kappa = 1.30 if free_surface else 1.05
    omega = kappa * c_max * math.sqrt(dims * abs(symbol_min(order))) / dx
    beta_sum = dims * beta0
    a_r = math.sqrt(2.0) * 0.5 * beta_sum
    a_i = math.sqrt(2.0) * omega
    centre = -0.5 * beta_sum
    gamma = 0.5 * (a_r + a_i)
    c0 = centre / gamma
    c1 = (a_r - a_i) / (a_r + a_i)
    return gamma, c0, c1


def faber_coefficients(dt, gamma, c0, c1, m, nodes=None):
    """a_0..a_m: trapezoid rule for (1/2pi) int exp(dt psi(e^{i th})) e^{-i j th} d th."""
    N = max(4 * m, 64) if nodes is None else nodes
    th = 2.0 * math.pi * np.arange(N) / N
    w = np.exp(1j * th)
    fvals = np.exp(dt * gamma * (w + c0 + c1 / w))
    a = np.empty(m + 1)
    for j in range(m + 1):
        a[j] = (np.sum(fvals * np.exp(-1j * j * th)) / N).real
    return a


def faber_step(model, U, src, t_n, dt, m, params, p=None):
    """One Faber step on the augmented state [U; e_p] (Sec. 3.2, Eq. matrix_ampli).

    ``params`` = (gamma, c0, c1).  ``src`` is a ``source.PointSource`` or ``None``.
    Returns the new U (the tail is reset to e_p, which is exact for the next step's
    re-expansion of f around t_{n+1}).
    """
    gamma, c0, c1 = params
    a = faber_coefficients(dt, gamma, c0, c1, m)
    if src is not None:
        p = src.p
        w = src.W(t_n, dt)
    else:
        p = 1 if p is None else p
        w = np.zeros(p)
    y0 = np.zeros(p)
    y0[-1] = 1.0

    def B(Ux, y):
        """F_1(H~) = H~/gamma - c0 I on [Ux; y]."""
        val = float(np.dot(w, y))
        HU = apply_H(model, Ux, None if src is None else (*src.node, val))
        Ty = tail_apply(y, dt)
        return (tuple(h / gamma - c0 * x for h, x in zip(HU, Ux)), Ty / gamma - c0 * y)

    P0 = (tuple(f.copy() for f in U), y0)
    acc = [a[0] * f for f in P0[0]]
    if m == 0:
        return tuple(acc)
    P1 = B(*P0)
    acc = [s + a[1] * f for s, f in zip(acc, P1[0])]
    prev, cur = P0, P1
    for j in range(2, m + 1):
        cj = 2.0 * c1 if j == 2 else c1
        BU, By = B(*cur)
        nxtU = tuple(b - cj * q for b, q in zip(BU, prev[0]))
        nxty = By - cj * prev[1]
        acc = [s + a[j] * f for s, f in zip(acc, nxtU)]
        prev, cur = cur, (nxtU, nxty)
    return tuple(acc)

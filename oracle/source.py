"""Ricker point source and the augmented source block of the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* The source f of Eq. (1) is a Ricker wavelet (Sec. 4.1) at one node, with delay t0
  (0.18 s at 15 Hz in Sec. 4.2).  Reading of the unstated discretisation: f = amp r(t)/dx^2
  added to the v-row at the nearest node, index floor(x/dx + 1/2) per axis (int32), and
  r(tau) = (1 - 2 a tau^2) exp(-a tau^2), a = pi^2 f_M^2, tau = t - t0.
* Augmented matrix of Eq. (matrix_ampli) (Sec. 3.2): H~ = [[H, W], [0, J]] with J the p x p
  upper shift and W's columns f and its derivatives, so that
  u(t) = [I 0] exp((t - t_n) H~) [u_n; e_p].  Reading: the derivatives are exact (Hermite
  recurrence of the Gaussian), and the tail is scaled by dt for conditioning -- tail
  operator J/dt and W column p-1-k = dt^k r^(k)(t_n) amp/dx^2 -- which is the same
  exponential after the change of variables y_{p-1-k} = (s/dt)^k / k!.

Pins: tests/test_oracle_integrators.py (derivatives against sympy's symbolic derivatives of
the closed form; the tail exponential reproduces the Taylor polynomial of f; the
nearest-node rule).
"""
import math

import numpy as np


def ricker(t, f_peak, t0):
    a = (math.pi * f_peak) ** 2
    tau = t - t0
    return (1.0 - 2.0 * a * tau * tau) * math.exp(-a * tau * tau)


def ricker_derivatives(t, f_peak, t0, p):
    """[r(t), r'(t), ..., r^(p-1)(t)] via r = -g''/(2a), g = exp(-a tau^2), and the Hermite
    recurrence g^(k) = -2 a tau g^(k-1) - 2 a (k-1) g^(k-2)."""
    a = (math.pi * f_peak) ** 2
    tau = t - t0
    g = [math.exp(-a * tau * tau)]
    g.append(-2.0 * a * tau * g[0])
    for k in range(2, p + 2):
        g.append(-2.0 * a * tau * g[k - 1] - 2.0 * a * (k - 1) * g[k - 2])
    return [-g[k + 2] / (2.0 * a) for k in range(p)]


def node_index(pos, dx):
    """Nearest node: floor(pos/dx + 1/2).  Raises for positions off the grid."""
    return int(math.floor(pos / dx + 0.5))


def source_node(model, sx, sy):
    i = node_index(sx, model.dx)
    j = node_index(sy, model.dx)
    if not (0 <= i < model.nx and 0 <= j < model.ny):
        raise ValueError("source outside the grid")
    return j, i


def W_scalars(t_n, dt, p, f_peak, t0, amp, dx):
    """Entries of W at the source node: W[p-1-k] = dt^k r^(k)(t_n) amp/dx^2."""
    r = ricker_derivatives(t_n, f_peak, t0, p)
    w = np.zeros(p)
    for k in range(p):
        w[p - 1 - k] = dt ** k * r[k] * amp / (dx * dx)
    return w


def tail_apply(y, dt):
    """(J/dt) y: (J y)_k = y_{k+1}, last entry 0."""
    out = np.zeros_like(y)
    out[:-1] = y[1:]
    return out / dt


def e_p(p):
    y = np.zeros(p)
    y[-1] = 1.0
    return y


class PointSource:
    """Source description for one shot: node, wavelet and amplitude."""

    def __init__(self, model, sx, sy, f_peak, t0, amp=1.0, p=12):
        self.j, self.i = source_node(model, sx, sy)
        self.f_peak, self.t0, self.amp, self.p = f_peak, t0, amp, p
        self.dx = model.dx

    @property
    def node(self):
        """Grid indices of the source node, slowest axis first."""
        return (self.j, self.i)

    def f(self, t):
        """f(t) value added at the source node's v entry (Eq. 1)."""
        return self.amp * ricker(t, self.f_peak, self.t0) / (self.dx * self.dx)

    def W(self, t_n, dt):
        return W_scalars(t_n, dt, self.p, self.f_peak, self.t0, self.amp, self.dx)


def apply_Htilde(model, U, y, src, w, dt, apply_H):
    """Augmented operator H~ [U; y] = [H U + e_src (w . y); (J/dt) y] (Eq. matrix_ampli)."""
    val = float(np.dot(w, y)) if src is not None else 0.0
    HU = apply_H(model, U, None if src is None else (*src.node, val))
    return HU, tail_apply(y, dt)

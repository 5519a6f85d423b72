"""Runge-Kutta integrators of the oracle: HORK (Sec. 3.2), RK3-2 and RK4-4 (Sec. 3.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* HORK (Sec. 3.2, after Gottlieb et al. 2003): k_0 = u^n; k_i = (I + dt H~) k_{i-1},
  i = 1..m-1; u^{n+1} = sum_{i=0}^{m-2} lambda_i k_i + lambda_{m-1} (I + dt H~) k_{m-1}.
  Reading of "straightforward" lambda: the linear SSP recursion lambda^(1) = [1];
  lambda^(m)_k = lambda^(m-1)_{k-1} / k (k = 1..m-2), lambda^(m)_{m-1} = 1/m!,
  lambda^(m)_0 = 1 - sum of the others.  Applied to the augmented H~ of Eq. (matrix_ampli).
* RK3-2 (Sec. 3.1, as printed): k1 = H u + f(t_n), k2 = H(u + dt/2 k1) + f(t_n + dt/2),
  k3 = H(u + dt/2 k2) + f(t_n + dt/2), u^{n+1} = u + dt k3.
* RK4-4 (Sec. 3.1, classical tableau; not printed in the paper): stages at t_n,
  t_n + dt/2 (twice), t_n + dt with weights 1/6, 1/3, 1/3, 1/6.

Pins: tests/test_oracle_integrators.py (HORK equals the degree-m Taylor polynomial of the dense
exp(dt H~); RK3-2 and RK4-4 equal their stability polynomials on a dense H and converge
at orders 2 and 4).
"""
from fractions import Fraction as Fr

import numpy as np

from .operator import apply_H
from .source import tail_apply


def hork_lambdas(m, exact=False):
    lam = [Fr(1)]
    for q in range(2, m + 1):
        new = [Fr(0)] * q
        for k in range(1, q - 1):
            new[k] = lam[k - 1] / k
        f = Fr(1)
        for i in range(2, q + 1):
            f *= i
        new[q - 1] = Fr(1) / f
        new[0] = 1 - sum(new[1:])
        lam = new
    return lam if exact else [float(x) for x in lam]


def _axpy(a, X, b, Y):
    return tuple(a * x + b * y for x, y in zip(X, Y))


def hork_step(model, U, src, t_n, dt, m, p=None):
    lam = hork_lambdas(m)
    if src is not None:
        p = src.p
        w = src.W(t_n, dt)
    else:
        p = 1 if p is None else p
        w = np.zeros(p)

    def step(Ux, y):
        """(I + dt H~) [Ux; y]."""
        val = float(np.dot(w, y))
        HU = apply_H(model, Ux, None if src is None else (*src.node, val))
        return _axpy(1.0, Ux, dt, HU), y + dt * tail_apply(y, dt)

    y = np.zeros(p)
    y[-1] = 1.0
    k = (tuple(f.copy() for f in U), y)
    acc = tuple(lam[0] * f for f in k[0]) if m >= 2 else None
    for i in range(1, m):
        k = step(*k)
        if i <= m - 2:
            acc = _axpy(1.0, acc, lam[i], k[0])
    last = step(*k)[0]
    if acc is None:
        return tuple(lam[m - 1] * f for f in last)
    return _axpy(1.0, acc, lam[m - 1], last)


def _Hf(model, X, src, t):
    return apply_H(model, X, None if src is None else (*src.node, src.f(t)))


def rk32_step(model, U, src, t_n, dt):
    k1 = _Hf(model, U, src, t_n)
    k2 = _Hf(model, _axpy(1.0, U, dt / 2, k1), src, t_n + dt / 2)
    k3 = _Hf(model, _axpy(1.0, U, dt / 2, k2), src, t_n + dt / 2)
    return _axpy(1.0, U, dt, k3)


def rk44_step(model, U, src, t_n, dt):
    k1 = _Hf(model, U, src, t_n)
    k2 = _Hf(model, _axpy(1.0, U, dt / 2, k1), src, t_n + dt / 2)
    k3 = _Hf(model, _axpy(1.0, U, dt / 2, k2), src, t_n + dt / 2)
    k4 = _Hf(model, _axpy(1.0, U, dt, k3), src, t_n + dt)
    return tuple(u + dt / 6.0 * (a + 2.0 * b + 2.0 * c + d)
                 for u, a, b, c, d in zip(U, k1, k2, k3, k4))

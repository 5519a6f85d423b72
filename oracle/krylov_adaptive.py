"""Adaptive Krylov exponential step (KIOPS-style dimension and substep control) of the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 3.2 uses the classical Arnoldi process with a fixed dimension m and one projection per
time step, and names adaptive schemes (KIOPS: adaptive substeps and cheaper bases) as the
improvement it leaves out (Secs. 3.2 and 6).  The paper gives no algorithm, so this module
is a reading built on two standard facts:

* Arnoldi relation and error estimate.  With A V_j = V_j H_j + h_{j+1,j} v_{j+1} e_j^T, the
  error of y(tau) = beta V_j exp(tau H_j) e_1 against exp(tau A) x is the series
      beta h_{j+1,j} sum_{k>=1} tau^k [phi_k(tau H_j)]_{j,1} A^{k-1} v_{j+1}
  (Saad, SIAM J. Numer. Anal. 29 (1992)), phi_0 = exp, phi_{k+1}(z) = (phi_k(z) - 1/k!)/z.
  Its first two terms bound the estimate
      err_j(tau) = beta h_{j+1,j} (tau |[phi_1(tau H_j)]_{j,1}|
                                   + tau^2 |[phi_2(tau H_j)]_{j,1}| |A v_{j+1}|),
  and exp(tau H_j) e_1, tau phi_1(tau H_j) e_1 and tau^2 phi_2(tau H_j) e_1 are the first
  three block columns of the top row of exp(tau [[H_j, e_1, 0], [0, 0, 1], [0, 0, 0]]) (one
  small exponential gives all three).  A v_{j+1} is the next basis vector's matvec, so it
  is reused when the basis grows.  The first term alone is the usual leading-order
  estimate; on the PML operator with its source column it ran 3-5x below the true error at
  whole-step tau, and the two-term sum 1.2-1.8x above it.
* Substeps compose: exp(A) x = exp(tau_K A) ... exp(tau_1 A) x with sum tau_k = 1.

Control (the reading): on the augmented A = dt H~_eta (as ``oracle.krylov.krylov_step``,
start vector [U; eta e_p]), each substep grows the basis one vector at a time, from m_min
to m_max.  It stops at the first j whose estimate meets err_j(tau) <= tol tau beta_k, with
beta_k the norm of the substep's start vector (error per unit of the normalised step, so
the whole step is held near tol relative to the augmented start vector; from U^n = 0 that
is the tail e_p, of norm 1).  If m_max vectors do not meet it,
tau shrinks by max(0.2, 0.9 (tol tau beta_k / err)^(1/m_max)) on the same basis (no new
matvecs).  After an accepted substep the next tau grows by min(2, 0.9 (tol tau beta_k /
err)^(1/j)), at most to the end of the step.  A happy breakdown (h_{j+1,j} <= breakdown_tol)
means the basis spans an invariant subspace, and the rest of the step is taken at once.
``window`` = q applies the incomplete orthogonalisation of ``oracle.krylov.arnoldi``.

Pins: tests/test_oracle_krylov_adaptive.py (phi_1 and phi_2 against their closed forms; the
dense exponential within the tolerance over a range of tolerances, windows and forced
substeps; the reduction to ``krylov_step`` at m_min = m_max with no error control; exact
results on an invariant subspace; the estimate against the true error).
"""
import numpy as np

from .krylov import expm
from .model import flatten, unflatten
from .operator import apply_H
from .source import tail_apply


def phi_block(Hj, tau):
    """(exp(tau H_j) e_1, tau phi_1(tau H_j) e_1, tau^2 phi_2(tau H_j) e_1) from one exponential
    of the twice-bordered matrix."""
    j = Hj.shape[0]
    B = np.zeros((j + 2, j + 2))
    B[:j, :j] = tau * Hj
    B[0, j] = tau
    B[j, j + 1] = tau
    E = expm(B)
    return E[:j, 0], E[:j, j], E[:j, j + 1]


def error_estimate(beta, h, ph1, ph2, anext):
    """err_j(tau) of the module header from the last entries of tau phi_1 e_1, tau^2 phi_2 e_1."""
    return beta * h * (abs(ph1[-1]) + abs(ph2[-1]) * anext)


def adaptive_exp(matvec, x, tol, m_min=1, m_max=30, window=None, breakdown_tol=1e-14,
                 tau0=1.0, max_rejections=60):
    """exp(A) x with A given by ``matvec``, under the control of the module header.

    Returns (result, info) with info = {"substeps", "matvecs", "dims", "taus"}."""
    if m_min < 1 or m_max < m_min:
        raise ValueError("need 1 <= m_min <= m_max")
    x = np.asarray(x, dtype=np.float64).copy()
    n = x.shape[0]
    s, tau = 0.0, min(1.0, tau0)
    info = {"substeps": 0, "matvecs": 0, "dims": [], "taus": []}

    def mv(v):
        info["matvecs"] += 1
        return matvec(v)

    while s < 1.0:
        tau = min(tau, 1.0 - s)
        beta = float(np.linalg.norm(x))
        if beta == 0.0:
            break
        V = np.zeros((n, m_max + 1))
        H = np.zeros((m_max + 1, m_max))
        V[:, 0] = x / beta
        accepted = None
        pending = None                 # A v_j, computed for the estimate at j - 1
        err = anext = 0.0
        for j in range(1, m_max + 1):
            w = mv(V[:, j - 1]) if pending is None else pending
            pending = None
            k0 = 0 if not window else max(0, j - window)
            for k in range(k0, j):
                H[k, j - 1] = float(np.dot(w, V[:, k]))
                w = w - H[k, j - 1] * V[:, k]
            H[j, j - 1] = float(np.linalg.norm(w))
            if H[j, j - 1] <= breakdown_tol:
                tau = 1.0 - s
                e, _, _ = phi_block(H[:j, :j], tau)
                accepted = (j, e, 0.0)
                break
            V[:, j] = w / H[j, j - 1]
            if j < m_min:
                continue
            pending = mv(V[:, j])
            anext = float(np.linalg.norm(pending))
            e, ph1, ph2 = phi_block(H[:j, :j], tau)
            err = error_estimate(beta, H[j, j - 1], ph1, ph2, anext)
            if err <= tol * tau * beta:
                accepted = (j, e, err)
                break
        if accepted is None:
            j = m_max
            for _ in range(max_rejections):
                tau *= max(0.2, 0.9 * (tol * tau * beta / err) ** (1.0 / m_max))
                e, ph1, ph2 = phi_block(H[:j, :j], tau)
                err = error_estimate(beta, H[j, j - 1], ph1, ph2, anext)
                if err <= tol * tau * beta:
                    accepted = (j, e, err)
                    break
            if accepted is None:
                raise RuntimeError("adaptive Krylov: substep did not meet the tolerance")
        j, e, err = accepted
        x = beta * (V[:, :j] @ e)
        s += tau
        info["substeps"] += 1
        info["dims"].append(j)
        info["taus"].append(tau)
        tau *= 2.0 if err == 0.0 else min(2.0, 0.9 * (tol * tau * beta / err) ** (1.0 / j))
    return x, info


def krylov_adaptive_step(model, U, src, t_n, dt, tol, m_min=1, m_max=30, window=None,
                         breakdown_tol=1e-14, tau0=1.0, p=None):
    """One step U^{n+1} = [I 0] exp(dt H~) [U^n; e_p] with the adaptive control above, on the
    same balanced augmented operator as ``oracle.krylov.krylov_step``.  Returns (U^{n+1}, info)."""
    if src is not None:
        p = src.p
        w = src.W(t_n, dt)
    else:
        p = 1 if p is None else p
        w = np.zeros(p)
    nU = model.n
    xu = flatten(U)
    eta = float(np.linalg.norm(xu))
    if eta == 0.0:
        eta = 1.0
    w = w / eta

    def matvec(x):
        Ux = unflatten(model, x[:nU])
        y = x[nU:]
        val = float(np.dot(w, y))
        HU = apply_H(model, Ux, None if src is None else (*src.node, val))
        return dt * np.concatenate([flatten(HU), tail_apply(y, dt)])

    y0 = np.zeros(p)
    y0[-1] = eta
    out, info = adaptive_exp(matvec, np.concatenate([xu, y0]), tol, m_min, m_max, window,
                             breakdown_tol, tau0)
    return unflatten(model, out[:nU]), info

"""Exact discrete adjoint of the oracle's Krylov step (reverse mode through Arnoldi).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Not in the paper: its Krylov integrator (Sec. 3.2) is forward only, and the inverse problem
that motivates an adjoint is named in its Secs. 3.3 and 6.  ``oracle.krylov.krylov_step`` maps
U^n to

    U^{n+1} = [I 0] beta V_m expm(H_m) e_1,

with modified Gram-Schmidt Arnoldi on A = dt H~_eta from x = [U^n; eta e_p], eta = |U^n|_2
(1 when U^n = 0) and W / eta in the source column of H~_eta.  The basis, the Hessenberg
matrix and eta all depend on U^n, so the step is not linear in U^n; it also depends on
m = c^2 through the v-row of H (Eq. 1): d(H x)_v / dm = L x_u + D x_w =: G(x).

This module differentiates that map itself, not the exponential it approximates: every
operation of the forward sweep is reversed in the opposite order.

* Output: y = beta (V e)_U with e = expm(H_m) e_1 gives
  beta_bar = ybar . V e, V_bar = beta ybar e^T, e_bar = beta V^T ybar and
  Hm_bar = L(H_m^T, e_bar e_1^T), where L(X, E) is the Frechet derivative of the
  exponential, read off the upper-right block of expm([[X, E], [0, X]]), and
  L(X, .)^* = L(X^T, .) under the Frobenius product.
* Arnoldi column j, backwards: v_{j+1} = w / h_{j+1,j} and h_{j+1,j} = |w| (when v_{j+1}
  is part of the basis), then the Gram-Schmidt updates w <- w - h_{kj} v_k with
  h_{kj} = w . v_k for k = j down to the first vector of the window, and finally
  w = A v_j, which sends A^T w_bar to v_j, dt w_bar_v * G(v_j) to dJ/dm, and
  -dt w_bar[source] (W . y_j) / eta^2 to eta_bar (y_j = the tail of v_j).
* Start: v_1 = x / beta, beta = |x|, x = [U; eta e_p], eta = |U| (when U != 0).

A happy breakdown is differentiated along the branch the forward sweep took.  The
transposes are independent of the CUDA path: H^T is the transposed sparse matrix of
``oracle.operator.assemble_H`` and the tail block's transpose is assembled column by column
from ``oracle.source.tail_apply``.

Pins: tests/test_oracle_krylov_adjoint.py (the taped sweep reproduces ``krylov_step``; one
step's adjoint against central differences of the step in U and in m; with a full-dimension
basis, the adjoint against the exact exponential transpose and against Van Loan's block
exponential; the FWI gradient against central differences of the Krylov misfit).
"""
import numpy as np

from .adjoint import G_of, misfit
from .krylov import expm
from .model import flatten, unflatten
from .operator import apply_H, assemble_H
from .source import tail_apply


def _tail_matrix(p, dt):
    """The p x p tail block J/dt, one column per unit vector."""
    T = np.zeros((p, p))
    for k in range(p):
        e = np.zeros(p)
        e[k] = 1.0
        T[:, k] = tail_apply(e, dt)
    return T


def expm_frechet(X, E):
    """L(X, E): upper-right block of expm([[X, E], [0, X]])."""
    n = X.shape[0]
    big = np.zeros((2 * n, 2 * n))
    big[:n, :n] = X
    big[:n, n:] = E
    big[n:, n:] = X
    return expm(big)[:n, n:]


class KrylovTape:
    """Forward Krylov step with every intermediate kept for the reverse sweep.

    Same operations, in the same order, as ``oracle.krylov.krylov_step``."""

    def __init__(self, model, U_flat, src, t_n, dt, m, p=None, breakdown_tol=1e-14,
                 window=None):
        self.model, self.src, self.dt, self.window = model, src, dt, window
        if src is not None:
            p = src.p
            w_raw = src.W(t_n, dt)
        else:
            p = 1 if p is None else p
            w_raw = np.zeros(p)
        self.p, self.w_raw = p, w_raw
        nU = model.n
        self.nU = nU
        U_flat = np.asarray(U_flat, dtype=np.float64)
        self.U = U_flat.copy()
        eta = float(np.linalg.norm(U_flat))
        self.eta_const = eta == 0.0
        self.eta = 1.0 if eta == 0.0 else eta
        self.w = w_raw / self.eta
        y0 = np.zeros(p)
        y0[-1] = self.eta
        x = np.concatenate([U_flat, y0])
        self.x = x
        beta = float(np.linalg.norm(x))
        self.beta = beta
        n = x.shape[0]
        V = np.zeros((n, m + 1))
        Hm = np.zeros((m + 1, m))
        self.ws = []          # per column j: [w before subtraction k0, ..., w after the last]
        self.k0 = []
        if beta == 0.0:
            self.V, self.Hm, self.m_eff = V[:, :0], Hm[:0, :0], 0
            self.out = np.zeros(nU)
            return
        V[:, 0] = x / beta
        m_eff = m
        for j in range(m):
            w = self.matvec(V[:, j])
            k0 = 0 if not window else max(0, j - window + 1)
            seq = [w]
            for k in range(k0, j + 1):
                Hm[k, j] = float(np.dot(w, V[:, k]))
                w = w - Hm[k, j] * V[:, k]
                seq.append(w)
            self.ws.append(seq)
            self.k0.append(k0)
            if j == m - 1:
                break
            Hm[j + 1, j] = float(np.linalg.norm(w))
            if Hm[j + 1, j] <= breakdown_tol:
                m_eff = j + 1
                break
            V[:, j + 1] = w / Hm[j + 1, j]
        self.V_full, self.H_full = V, Hm
        self.V, self.Hm, self.m_eff = V[:, :m_eff], Hm[:m_eff, :m_eff], m_eff
        self.e = expm(self.Hm)[:, 0]
        self.out = beta * (self.V[:nU] @ self.e)

    def matvec(self, x):
        m, nU = self.model, self.nU
        Ux = unflatten(m, x[:nU])
        y = x[nU:]
        val = float(np.dot(self.w, y))
        HU = apply_H(m, Ux, None if self.src is None else (*self.src.node, val))
        return self.dt * np.concatenate([flatten(HU), tail_apply(y, self.dt)])


def krylov_exact_adjoint_step(model, U_prev_flat, ybar, src, t_n, dt, m, HT=None,
                              window=None, breakdown_tol=1e-14, p=None):
    """Cotangent of U^{n-1} and the m-gradient of one Krylov step, by reverse mode through
    the step (see the module header).  ``ybar``: dJ/dU^n (flat).  Returns (Ubar, grad [ny*nx])."""
    tp = KrylovTape(model, U_prev_flat, src, t_n, dt, m, p=p, breakdown_tol=breakdown_tol,
                    window=window)
    nU, p = tp.nU, tp.p
    nu = model.nx * model.ny
    grad = np.zeros(nu)
    if tp.m_eff == 0:
        return np.zeros(nU), grad
    if HT is None:
        HT = assemble_H(model).T.tocsr()
    TT = _tail_matrix(p, dt).T
    src_v = None if src is None else nu + src.node[0] * model.nx + src.node[1]
    me = tp.m_eff
    V, Hm = tp.V_full, tp.H_full
    ybar_full = np.concatenate([np.asarray(ybar, dtype=np.float64), np.zeros(p)])

    # output y = beta (V e)_U
    Ve = V[:, :me] @ tp.e
    beta_bar = float(ybar_full @ Ve)
    Vbar = np.zeros_like(V)
    Vbar[:, :me] = tp.beta * np.outer(ybar_full, tp.e)
    e_bar = tp.beta * (V[:, :me].T @ ybar_full)
    Ebar = np.zeros((me, me))
    Ebar[:, 0] = e_bar
    Hbar = np.zeros_like(Hm)
    Hbar[:me, :me] = expm_frechet(tp.Hm.T, Ebar)
    eta_bar = 0.0

    for j in range(me - 1, -1, -1):
        seq, k0 = tp.ws[j], tp.k0[j]
        w_last = seq[-1]
        if j < me - 1:
            h = Hm[j + 1, j]
            wbar = Vbar[:, j + 1] / h
            hbar = Hbar[j + 1, j] - float(Vbar[:, j + 1] @ w_last) / (h * h)
            wbar = wbar + hbar * w_last / h
        else:
            wbar = np.zeros_like(w_last)
        for idx, k in reversed(list(enumerate(range(k0, j + 1)))):
            w_before = seq[idx]
            hk = Hm[k, j]
            hkbar = Hbar[k, j] - float(wbar @ V[:, k])
            Vbar[:, k] -= hk * wbar
            wbar = wbar + hkbar * V[:, k]
            Vbar[:, k] += hkbar * w_before
        # w = A v_j
        vj = V[:, j]
        wU, wy = wbar[:nU], wbar[nU:]
        back = np.empty_like(vj)
        back[:nU] = dt * (HT @ wU)
        back[nU:] = dt * (TT @ wy)
        if src_v is not None:
            back[nU:] += dt * tp.w * wU[src_v]
            eta_bar -= dt * wU[src_v] * float(tp.w_raw @ vj[nU:]) / (tp.eta * tp.eta)
        Vbar[:, j] += back
        grad += dt * wU[nu:2 * nu] * G_of(model, vj[:nU])

    # v_1 = x / beta, beta = |x|
    x, beta = tp.x, tp.beta
    xbar = Vbar[:, 0] / beta
    beta_bar -= float(Vbar[:, 0] @ x) / (beta * beta)
    xbar = xbar + beta_bar * x / beta
    Ubar = xbar[:nU].copy()
    eta_bar += xbar[nU + p - 1]
    if not tp.eta_const:
        Ubar += eta_bar * tp.U / tp.eta
    return Ubar, grad


def krylov_exact_fwi_gradient(model, shots, d_obs, dt, nsteps, m, window=None):
    """dJ/dm (m = c^2 at the nodes, [ny, nx]) of the Krylov misfit by the exact discrete
    adjoint; the forward is ``krylov_step`` (through ``KrylovTape``).  Returns (J, grad)."""
    HT = assemble_H(model).T.tocsr()
    nu = model.nx * model.ny
    grad = np.zeros(nu)
    seis = []
    for (src, rec_nodes), D in zip(shots, d_obs):
        U = np.zeros(model.n)
        Us, S = [U], []
        for n in range(nsteps):
            U = KrylovTape(model, U, src, n * dt, dt, m, window=window).out
            Us.append(U)
            S.append(unflatten(model, U)[0][rec_nodes[:, 0], rec_nodes[:, 1]].copy())
        S = np.array(S)
        seis.append(S)
        r = S - D
        ridx = rec_nodes[:, 0] * model.nx + rec_nodes[:, 1]
        lam = np.zeros(model.n)
        np.add.at(lam, ridx, r[nsteps - 1])
        for n in range(nsteps, 0, -1):
            lam, g = krylov_exact_adjoint_step(model, Us[n - 1], lam, src, (n - 1) * dt, dt, m,
                                               HT, window=window)
            grad += g
            if n - 1 >= 1:
                np.add.at(lam, ridx, r[n - 2])
    return misfit(seis, d_obs), grad.reshape(model.ny, model.nx)

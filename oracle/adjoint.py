"""Discrete adjoint of the Faber time stepping and the FWI gradient (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Not in the paper (its Secs. 3.3 and 6 motivate it: the inverse problem stores one state per
time step, N_mem = T/dt).  Misfit J(m) = 1/2 sum_n |R U^n - d^n|^2 over the seismogram
samples n = 1..N (R picks u at the receivers), m = c^2 at the nodes.  U^n = Phi_n(U^{n-1})
is one Faber step (oracle.faber): p_0 = [U^{n-1}; e_p], p_1 = B p_0, p_2 = B p_1 - 2 c1 p_0,
p_j = B p_{j-1} - c1 p_{j-2}, U^n = sum_j a_j p_j (U part), B = H~/gamma - c0 I.

Reverse recurrence for a cotangent ybar of U^n (q_j = dJ/dp_j, U parts only -- the tail's
cotangent never feeds back into U because H~ is block upper triangular):
    q_m = a_m ybar,  q_{j-1} = a_{j-1} ybar + B^T q_j - c'_{j+1} q_{j+1}
with c'_2 = 2 c1, c'_k = c1 (k >= 3), q_{m+1} = 0; the cotangent of U^{n-1} is q_0.
m enters only the v-row of H (Eq. 1): d(H x)_v / dm = L x_u + D x_w (the Laplacian and the
divergence of w), so dJ/dm += (1/gamma) sum_{j=1..m} q_{j,v} * G(p_{j-1}), G(x) = L x_u + D x_w.
Time loop: lambda^N = R^T r^N, lambda^{n-1} = q_0(lambda^n) + R^T r^{n-1}.

HORK (Sec. 3.2) is handled the same way: u^{n+1} = sum_i w_i k_i, k_i = (I + dt H~) k_{i-1}
with w_i the lambda weights; r_m = w_m ybar, r_{i-1} = w_{i-1} ybar + (I + dt H)^T r_i and
dJ/dm += dt sum_i r_{i,v} G(k_{i-1}).

Krylov (Sec. 3.2) is not linear in u^n (the Arnoldi basis depends on it), so its adjoint is
the step-level linearisation of U^{n+1} = [I 0] exp(dt H~) [U^n; e_p] (the reading of the
Krylov row of the FWI gradient): the cotangent of U^n is exp(dt H)^T ybar, computed by
Arnoldi on dt H^T from ybar; the m-gradient is the Frechet integral
    dJ/dm += int_0^dt [exp((dt - s) H)^T ybar]_v  G(x(s)) ds,   x(s) = [I 0] exp(s H~)[U^n; e_p],
evaluated by 4-point Gauss-Legendre on [0, dt], with x(s) and the adjoint states taken as
dense output of the forward and adjoint Arnoldi bases (exp(tau A) x ~ |x| V exp(tau H_m) e_1).

This route is independent of the CUDA path: B^T uses the transposed sparse matrix of
``oracle.operator.assemble_H``.  Pins: tests/test_oracle_adjoint.py (dot-product identity
of one adjoint step; central finite differences of J along seeded directions; the Krylov
dense states against dense expm of the augmented matrix at the Gauss nodes).
"""
import math

import numpy as np

from .faber import faber_coefficients
from .model import flatten, unflatten
from .operator import apply_H, assemble_H, dx_node, dxx, dy_node, dyy
from .source import tail_apply


def G_of(model, x_flat):
    """G(x) = L x_u + D x_w at the nodes (flattened [ny*nx])."""
    u, _v, wx, wy = unflatten(model, x_flat)
    g = dxx(model, u) + dyy(model, u) + dx_node(model, wx) + dy_node(model, wy)
    return g.ravel()


def faber_tape(model, U_flat, src, t_n, dt, m, params):
    """Forward Faber step keeping p_0..p_m (U parts).  Returns (tape list, U^{n+1})."""
    gamma, c0, c1 = params
    a = faber_coefficients(dt, gamma, c0, c1, m)
    p = src.p if src is not None else 1
    w = src.W(t_n, dt) if src is not None else np.zeros(p)
    nU = model.n

    def B(x, y):
        val = float(np.dot(w, y))
        HU = apply_H(model, unflatten(model, x), None if src is None else (src.j, src.i, val))
        return flatten(HU) / gamma - c0 * x, tail_apply(y, dt) / gamma - c0 * y

    y0 = np.zeros(p)
    y0[-1] = 1.0
    tape = [U_flat.copy()]
    tails = [y0]
    if m >= 1:
        x1, y1 = B(U_flat, y0)
        tape.append(x1)
        tails.append(y1)
    for j in range(2, m + 1):
        cj = 2.0 * c1 if j == 2 else c1
        bx, by = B(tape[-1], tails[-1])
        tape.append(bx - cj * tape[-2])
        tails.append(by - cj * tails[-2])
    out = sum(a[j] * tape[j] for j in range(m + 1))
    return tape, out


def faber_adjoint_step(model, U_prev_flat, ybar, src, t_n, dt, m, params, HT=None):
    """Cotangent of U^{n-1} and the gradient contribution of one Faber step.

    ``ybar``: dJ/dU^n (flat).  Returns (q_0, grad_m [ny*nx])."""
    gamma, c0, c1 = params
    a = faber_coefficients(dt, gamma, c0, c1, m)
    tape, _ = faber_tape(model, U_prev_flat, src, t_n, dt, m, params)
    if HT is None:
        HT = assemble_H(model).T.tocsr()
    nu = model.nx * model.ny

    def BT(q):
        return (HT @ q) / gamma - c0 * q

    def cprime(k):
        return 0.0 if k <= 1 else (2.0 * c1 if k == 2 else c1)

    grad = np.zeros(nu)
    q_next = np.zeros_like(ybar)                  # q_{j+1}
    q_cur = a[m] * ybar                           # q_m
    for j in range(m, 0, -1):
        grad += (1.0 / gamma) * q_cur[nu:2 * nu] * G_of(model, tape[j - 1])
        q_prev = a[j - 1] * ybar + BT(q_cur) - cprime(j + 1) * q_next
        q_next, q_cur = q_cur, q_prev
    return q_cur, grad


def hork_weights(m):
    """Weights w_i of u^{n+1} = sum_{i=0}^{m} w_i k_i for HORK (Sec. 3.2): w_i = lambda_i
    (i <= m-2), w_{m-1} = 0, w_m = lambda_{m-1}."""
    from .rk import hork_lambdas
    lam = hork_lambdas(m)
    w = [0.0] * (m + 1)
    for i in range(m + 1):
        w[i] = lam[i] if i <= m - 2 else (0.0 if i == m - 1 else lam[m - 1])
    return w


def hork_tape(model, U_flat, src, t_n, dt, m):
    """k_0 = [U; e_p], k_i = (I + dt H~) k_{i-1}; returns (k_0..k_m U parts, U^{n+1})."""
    p = src.p if src is not None else 1
    w = src.W(t_n, dt) if src is not None else np.zeros(p)
    y = np.zeros(p)
    y[-1] = 1.0
    ks = [U_flat.copy()]
    x = U_flat.copy()
    for _ in range(m):
        val = float(np.dot(w, y))
        HU = apply_H(model, unflatten(model, x), None if src is None else (src.j, src.i, val))
        x = x + dt * flatten(HU)
        y = y + dt * tail_apply(y, dt)
        ks.append(x)
    wt = hork_weights(m)
    return ks, sum(wt[i] * ks[i] for i in range(m + 1))


def hork_adjoint_step(model, U_prev_flat, ybar, src, t_n, dt, m, HT=None):
    """Cotangent of U^{n-1} and the gradient contribution of one HORK step:
    r_m = w_m ybar, r_{i-1} = w_{i-1} ybar + (I + dt H)^T r_i, grad += dt r_{i,v} G(k_{i-1})."""
    ks, _ = hork_tape(model, U_prev_flat, src, t_n, dt, m)
    if HT is None:
        HT = assemble_H(model).T.tocsr()
    wt = hork_weights(m)
    nu = model.nx * model.ny
    grad = np.zeros(nu)
    r = wt[m] * ybar
    for i in range(m, 0, -1):
        grad += dt * r[nu:2 * nu] * G_of(model, ks[i - 1])
        r = wt[i - 1] * ybar + r + dt * (HT @ r)
    return r, grad


def gauss_legendre4():
    """Nodes and weights of the 4-point Gauss-Legendre rule on [0, 1] (exact for degree 7):
    nodes (1 +- sqrt(3/7 -+ (2/7) sqrt(6/5))) / 2, weights (18 +- sqrt(30)) / 72."""
    a = math.sqrt(3.0 / 7.0 - 2.0 / 7.0 * math.sqrt(6.0 / 5.0))
    b = math.sqrt(3.0 / 7.0 + 2.0 / 7.0 * math.sqrt(6.0 / 5.0))
    wa, wb = (18.0 + math.sqrt(30.0)) / 36.0, (18.0 - math.sqrt(30.0)) / 36.0
    x = np.array([-b, -a, a, b])
    w = np.array([wb, wa, wa, wb])
    return (1.0 + x) / 2.0, w / 2.0


def krylov_dense_states(model, U_prev_flat, src, t_n, dt, m, taus=None):
    """Dense output of one Krylov step (Sec. 3.2): x(tau dt) = [I 0] beta V_m exp(tau H_m) e_1,
    the grid part of the Arnoldi approximation of exp(tau dt H~)[U; e_p] from the step's own
    basis (start vector [U; eta e_p], W / eta, as krylov_step), at the 4-point Gauss-Legendre
    nodes on [0, 1] unless taus is given.  Returns a list of flat state vectors."""
    from .krylov import arnoldi, expm
    nU = model.n
    p = src.p if src is not None else 1
    w = src.W(t_n, dt) if src is not None else np.zeros(p)
    eta = float(np.linalg.norm(U_prev_flat))
    eta = eta if eta > 0.0 else 1.0
    w = w / eta

    def matvec(x):
        Ux = unflatten(model, x[:nU])
        val = float(np.dot(w, x[nU:]))
        HU = apply_H(model, Ux, None if src is None else (*src.node, val))
        return dt * np.concatenate([flatten(HU), tail_apply(x[nU:], dt)])

    y0 = np.zeros(p)
    y0[-1] = eta
    beta, V, Hm, _ = arnoldi(matvec, np.concatenate([U_prev_flat, y0]), m)
    if taus is None:
        taus = gauss_legendre4()[0]
    return [beta * (V[:nU] @ expm(tau * Hm)[:, 0]) if beta > 0.0 else np.zeros(nU) for tau in taus]


def krylov_adjoint_step(model, U_prev_flat, ybar, src, t_n, dt, m, HT=None):
    """Cotangent of U^{n-1} and the m-gradient of one Krylov step (linearised, see the module
    header).  Returns (exp(dt H)^T ybar by Arnoldi, grad [ny*nx])."""
    from .krylov import arnoldi, expm
    nU = model.n
    nu = model.nx * model.ny
    if HT is None:
        HT = assemble_H(model).T.tocsr()
    taus, wts = gauss_legendre4()
    # forward states x(tau_q dt): dense output of the step's own Arnoldi basis
    xs = krylov_dense_states(model, U_prev_flat, src, t_n, dt, m, taus)
    # adjoint Arnoldi on dt H^T from ybar
    beta_t, Vt, Ht, _ = arnoldi(lambda y: dt * (HT @ y), ybar, m)

    def adj(sig):
        return beta_t * (Vt @ expm(sig * Ht)[:, 0]) if beta_t > 0.0 else np.zeros(nU)

    grad = np.zeros(nu)
    for x, tau, wq in zip(xs, taus, wts):
        grad += dt * wq * adj(1.0 - tau)[nu:2 * nu] * G_of(model, x)
    return adj(1.0), grad


def faber_forward(model, shots, dt, nsteps, m, params, U0=None, method="faber"):
    """Forward simulation of every shot; returns (states per shot [N+1 flat], seismograms)."""
    states, seis = [], []
    for src, rec_nodes in shots:
        U = np.zeros(model.n) if U0 is None else U0.copy()
        Us = [U]
        S = []
        for n in range(nsteps):
            if method == "faber":
                _, U = faber_tape(model, U, src, n * dt, dt, m, params)
            elif method == "krylov":
                from .krylov import krylov_step
                U = flatten(krylov_step(model, unflatten(model, U), src, n * dt, dt, m))
            else:
                _, U = hork_tape(model, U, src, n * dt, dt, m)
            Us.append(U)
            S.append(unflatten(model, U)[0][rec_nodes[:, 0], rec_nodes[:, 1]].copy())
        states.append(Us)
        seis.append(np.array(S))
    return states, seis


def misfit(seis, d_obs):
    return 0.5 * sum(float(np.sum((s - d) ** 2)) for s, d in zip(seis, d_obs))


def fwi_gradient(model, shots, d_obs, dt, nsteps, m, params, method="faber"):
    """dJ/dm (m = c^2 at the nodes, [ny, nx]) by the discrete adjoint; returns (J, grad)."""
    states, seis = faber_forward(model, shots, dt, nsteps, m, params, method=method)
    HT = assemble_H(model).T.tocsr()
    nu = model.nx * model.ny
    grad = np.zeros(nu)
    for (src, rec_nodes), Us, S, D in zip(shots, states, seis, d_obs):
        r = S - D                                   # residuals [N, nrec]
        lam = np.zeros(model.n)
        ridx = rec_nodes[:, 0] * model.nx + rec_nodes[:, 1]
        np.add.at(lam, ridx, r[nsteps - 1])
        for n in range(nsteps, 0, -1):
            if method == "faber":
                q0, g = faber_adjoint_step(model, Us[n - 1], lam, src, (n - 1) * dt, dt, m, params, HT)
            elif method == "krylov":
                q0, g = krylov_adjoint_step(model, Us[n - 1], lam, src, (n - 1) * dt, dt, m, HT)
            else:
                q0, g = hork_adjoint_step(model, Us[n - 1], lam, src, (n - 1) * dt, dt, m, HT)
            grad += g
            lam = q0
            if n - 1 >= 1:
                np.add.at(lam, ridx, r[n - 2])
    return misfit(seis, d_obs), grad.reshape(model.ny, model.nx)


def checkpoint_stride(nsteps, budget):
    """Store every stride-th state so that at most ``budget`` are kept (checkpoint-schedule
    reading; the paper only counts stored states, N_mem = T/dt): stride 1 when
    nsteps <= budget, else ceil(nsteps / budget)."""
    if nsteps <= budget:
        return 1
    return -(-nsteps // budget)

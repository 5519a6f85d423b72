"""Krylov/Arnoldi exponential integrator (Sec. 3.2, "Krylov subspace projection") of the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Arnoldi (the listing of Sec. 3.2), modified Gram-Schmidt order: v_1 = x/|x|;
for j = 1..m: w = A v_j; for k = 1..j: h_{k,j} = w . v_k, w = w - h_{k,j} v_k;
h_{j+1,j} = |w|; v_{j+1} = w / h_{j+1,j}.  Then exp(A) x ~ |x| V_m exp(H_m) e_1.

Readings: the index garble "A_{i,j}" inside the inner loop is read A_{k,j}; the method is
applied to A = dt H~ acting on [u^n; e_p] (Eq. matrix_ampli), so time is absorbed in the
matrix; exactly m matrix-vector products are taken and the top m x m block of the
Hessenberg matrix is exponentiated (h_{m+1,m} and v_{m+1} do not enter the result); a
happy breakdown (h_{j+1,j} <= ``breakdown_tol``) stops the process with m_eff = j.
The augmented tail is balanced against the wavefield: the start vector is [u^n; eta e_p]
with W / eta in place of W, eta = |u^n|_2 (1 if u^n = 0).  The exact exponential does not
depend on eta (the tail block is linear), but a tail of norm 1 beside a wavefield of norm
1e-7 makes the final combination cancel O(1) terms down to the 1e-7 result.

The small exponential ("Pade" in Sec. 3.2, degree unstated) is the [13/13] Pade
approximant with scaling and squaring (Higham, SIAM J. Matrix Anal. Appl. 26 (2005)),
written here from the published method: Pade coefficients from their closed form,
s = max(0, ceil(log2(|A|_1 / theta_13))), theta_13 = 5.371920351148152.

Pins: tests/test_oracle_integrators.py (expm against scipy.linalg.expm and closed forms; with
m = n the step reproduces the dense exponential; orthonormality of the basis).
"""
import math

import numpy as np

from .model import flatten, unflatten
from .operator import apply_H
from .source import tail_apply

THETA13 = 5.371920351148152


def pade_coefficients(q):
    """b_k = (2q-k)! q! / ((2q)! k! (q-k)!), k = 0..q: numerator of the [q/q] Pade of exp."""
    f = math.factorial
    return [f(2 * q - k) * f(q) / (f(2 * q) * f(k) * f(q - k)) for k in range(q + 1)]


def expm(A):
    """Matrix exponential by [13/13] Pade with scaling and squaring."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if n == 0:
        return A.copy()
    b = pade_coefficients(13)
    norm1 = np.abs(A).sum(axis=0).max()
    s = 0 if norm1 <= THETA13 else int(math.ceil(math.log2(norm1 / THETA13)))
    A = A / (2.0 ** s)
    I = np.eye(n)
    A2 = A @ A
    A4 = A2 @ A2
    A6 = A4 @ A2
    U = A @ (A6 @ (b[13] * A6 + b[11] * A4 + b[9] * A2) + b[7] * A6 + b[5] * A4 + b[3] * A2
             + b[1] * I)
    V = A6 @ (b[12] * A6 + b[10] * A4 + b[8] * A2) + b[6] * A6 + b[4] * A4 + b[2] * A2 + b[0] * I
    R = np.linalg.solve(V - U, V + U)
    for _ in range(s):
        R = R @ R
    return R


def arnoldi(matvec, x, m, breakdown_tol=1e-14, window=None):
    """MGS Arnoldi.  Returns (beta, V (n x m_eff), Hm (m_eff x m_eff), m_eff).

    ``window`` = q: incomplete orthogonalisation (each new vector against the q most recent
    basis vectors only; the library's option for cutting the Gram-Schmidt cost)."""
    beta = float(np.linalg.norm(x))
    n = x.shape[0]
    V = np.zeros((n, m + 1))
    Hm = np.zeros((m + 1, m))
    if beta == 0.0:
        return 0.0, V[:, :0], Hm[:0, :0], 0
    V[:, 0] = x / beta
    m_eff = m
    for j in range(m):
        w = matvec(V[:, j])
        k0 = 0 if not window else max(0, j - window + 1)
        for k in range(k0, j + 1):
            Hm[k, j] = float(np.dot(w, V[:, k]))
            w = w - Hm[k, j] * V[:, k]
        if j == m - 1:
            break
        Hm[j + 1, j] = float(np.linalg.norm(w))
        if Hm[j + 1, j] <= breakdown_tol:
            m_eff = j + 1
            break
        V[:, j + 1] = w / Hm[j + 1, j]
    return beta, V[:, :m_eff], Hm[:m_eff, :m_eff], m_eff


def krylov_step(model, U, src, t_n, dt, m, p=None, breakdown_tol=1e-14, return_info=False,
                window=None):
    """One Krylov step: [I 0] exp(dt H~) [U; e_p] by Arnoldi with m matvecs (``window``: the
    incomplete-orthogonalisation option of ``arnoldi``)."""
    if src is not None:
        p = src.p
        w = src.W(t_n, dt)
    else:
        p = 1 if p is None else p
        w = np.zeros(p)
    nU = model.n

    def matvec(x):
        Ux = unflatten(model, x[:nU])
        y = x[nU:]
        val = float(np.dot(w, y))
        HU = apply_H(model, Ux, None if src is None else (*src.node, val))
        Ty = tail_apply(y, dt)
        return dt * np.concatenate([flatten(HU), Ty])

    xu = flatten(U)
    eta = float(np.linalg.norm(xu))
    if eta == 0.0:
        eta = 1.0
    w = w / eta
    y0 = np.zeros(p)
    y0[-1] = eta
    x = np.concatenate([xu, y0])
    beta, V, Hm, m_eff = arnoldi(matvec, x, m, breakdown_tol, window)
    if m_eff == 0:
        out = unflatten(model, np.zeros(nU))
    else:
        e = expm(Hm)[:, 0]
        out = unflatten(model, beta * (V[:nU] @ e))
    return (out, m_eff) if return_info else out

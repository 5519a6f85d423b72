"""Discrete adjoint of the leap-frog scheme and the FWI gradient through it (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The scheme is Sec. 3.1's two-step method as read in ``oracle.leapfrog`` (averaged damping of
w).  One step maps z^n = (u^n, u^{n-1}, w^n, w^{n-1}), w = (w_x, w_y) in ``flatten`` order,
linearly:

    u^{n+1} = s (2u^n/dt^2 + (b/(2dt) - 1/dt^2) u^{n-1} + H_vu u^n + H_vw w^n + f(t_n) e_src),
              s = 1 / (1/dt^2 + b/(2dt)),  b = b_x + b_y at the nodes;
    w^{n+1} = ((1 - beta dt) w^{n-1} + 2 dt H_wu u^n) / (1 + beta dt),  beta = -diag(H_ww),

where H_vu, H_vw, H_wu and H_ww are blocks of the independently assembled H of Eq. 1
(``oracle.operator.assemble_H``): the v row of H without its -b v term is the leap-frog
right-hand side, and the w rows are the w equations.  The misfit is J = 1/2 sum_n
|R u^{n+1} - d^n|^2 with m = c^2 at the nodes; the adjoint runs backward with A^T, and each
step adds s (L u^n + D w^n) lambda_u^{n+1} to dJ/dm.

Pins: tests/test_oracle_leapfrog_adjoint.py (the assembled step equals ``leapfrog_step``;
the gradient equals central differences of J computed with ``leapfrog_step``).
"""
import numpy as np
import scipy.sparse as sp

from .model import flatten, unflatten
from .operator import assemble_H, dx_node, dxx, dy_node, dyy


def _blocks(model):
    H = assemble_H(model).tocsr()
    nu = model.nx * model.ny
    n = model.n
    return (H[nu:2 * nu, :nu], H[nu:2 * nu, 2 * nu:n], H[2 * nu:n, :nu],
            -H[2 * nu:n, 2 * nu:n].diagonal())


def step_matrix(model, dt):
    """A (sparse) with z^{n+1} = A z^n for the source-free step, and s (for the source and the
    gradient)."""
    Hvu, Hvw, Hwu, beta = _blocks(model)
    nu = model.nx * model.ny
    nw = model.n - 2 * nu
    b = (model.beta_x_node()[None, :] + model.beta_y_node()[:, None]).ravel()
    s = 1.0 / (1.0 / dt ** 2 + b / (2.0 * dt))
    S = sp.diags(s)
    I_u = sp.identity(nu, format="csr")
    I_w = sp.identity(nw, format="csr")
    Dinv = sp.diags(1.0 / (1.0 + beta * dt))
    row_u = [S @ (2.0 / dt ** 2 * I_u + Hvu), S @ sp.diags(b / (2.0 * dt) - 1.0 / dt ** 2), S @ Hvw, None]
    row_um = [I_u, None, None, None]
    row_w = [2.0 * dt * (Dinv @ Hwu), None, None, Dinv @ sp.diags(1.0 - beta * dt)]
    row_wm = [None, None, I_w, None]
    A = sp.bmat([row_u, row_um, row_w, row_wm], format="csr")
    return A, s


def pack(model, LF):
    """z from the leap-frog tuple (u, u^{n-1}, w_x, w_x^{n-1}, w_y, w_y^{n-1})."""
    u, um, wx, wxm, wy, wym = LF
    return np.concatenate([u.ravel(), um.ravel(), wx.ravel(), wy.ravel(), wxm.ravel(), wym.ravel()])


def unpack(model, z):
    nu = model.nx * model.ny
    nx_w = model.ny * (model.nx - 1)
    nw = model.n - 2 * nu
    u, um = z[:nu].reshape(model.ny, model.nx), z[nu:2 * nu].reshape(model.ny, model.nx)
    w, wm = z[2 * nu:2 * nu + nw], z[2 * nu + nw:]
    sh_x, sh_y = (model.ny, model.nx - 1), (model.ny - 1, model.nx)
    return (u, um, w[:nx_w].reshape(sh_x), wm[:nx_w].reshape(sh_x), w[nx_w:].reshape(sh_y),
            wm[nx_w:].reshape(sh_y))


def _G(model, u, wx, wy):
    """L u + D w at the nodes (the derivative of the leap-frog right-hand side w.r.t. c^2)."""
    return dxx(model, u) + dyy(model, u) + dx_node(model, wx) + dy_node(model, wy)


def forward(model, shots, dt, nsteps):
    """Every shot from rest; returns (states z^0..z^N per shot, seismograms [N, nrec])."""
    A, s = step_matrix(model, dt)
    nu = model.nx * model.ny
    states, seis = [], []
    for src, rec_nodes in shots:
        z = np.zeros(A.shape[0])
        zs, S = [z], []
        k = src.j * model.nx + src.i
        for n in range(nsteps):
            z = A @ z
            z[k] += s[k] * src.f(n * dt)
            zs.append(z)
            S.append(z[:nu].reshape(model.ny, model.nx)[rec_nodes[:, 0], rec_nodes[:, 1]].copy())
        states.append(zs)
        seis.append(np.array(S))
    return states, seis


def fwi_gradient(model, shots, d_obs, dt, nsteps):
    """(J, dJ/dm [ny, nx]) through the leap-frog scheme by its discrete adjoint."""
    A, s = step_matrix(model, dt)
    AT = A.T.tocsr()
    nu = model.nx * model.ny
    states, seis = forward(model, shots, dt, nsteps)
    grad = np.zeros(nu)
    J = 0.0
    for (src, rec_nodes), zs, S, D in zip(shots, states, seis, d_obs):
        r = S - D
        J += 0.5 * float(np.sum(r * r))
        ridx = rec_nodes[:, 0] * model.nx + rec_nodes[:, 1]
        lam = np.zeros(A.shape[0])
        np.add.at(lam, ridx, r[nsteps - 1])
        for n in range(nsteps - 1, -1, -1):
            u, _, wx, _, wy, _ = unpack(model, zs[n])
            grad += s * _G(model, u, wx, wy).ravel() * lam[:nu]
            lam = AT @ lam
            if n >= 1:
                np.add.at(lam, ridx, r[n - 1])
    return J, grad.reshape(model.ny, model.nx)

"""Time loops, receivers and error measures of the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Seismogram (Sec. 5.1): u sampled at the receiver nodes after every step; receiver node
  indices use the nearest-node rule of ``oracle.source.node_index``.
* Error (Secs. 4.2 and 5.2; the norm is unstated): relative L2,
  |s - s_ref|_2 / |s_ref|_2 over all receivers and samples.
* Methods: "faber", "krylov", "hork" (degree / dimension / stages m), "rk32", "rk44",
  "leapfrog".

Parity status: the loop is bookkeeping around the pinned step functions.
"""
import numpy as np

from .faber import ellipse_params, faber_step
from .krylov import krylov_step
from .leapfrog import leapfrog_init, leapfrog_step
from .rk import hork_step, rk32_step, rk44_step
from .source import node_index


def receiver_nodes(model, rec):
    out = []
    for x, y in rec:
        i, j = node_index(x, model.dx), node_index(y, model.dx)
        if not (0 <= i < model.nx and 0 <= j < model.ny):
            raise ValueError("receiver outside the grid")
        out.append((j, i))
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def record(U_u, rec_nodes):
    return U_u[rec_nodes[:, 0], rec_nodes[:, 1]].copy()


def rel_l2(s, s_ref):
    s = np.asarray(s, dtype=np.float64)
    s_ref = np.asarray(s_ref, dtype=np.float64)
    den = np.linalg.norm(s_ref)
    return float(np.linalg.norm(s - s_ref) / den) if den > 0 else float(np.linalg.norm(s))


def run(model, method, dt, nsteps, src=None, rec_nodes=None, m=None, U0=None, t0=0.0,
        faber_params=None, lf_variant="averaged"):
    """Advance ``nsteps`` steps; return (final U, seismogram [nsteps, nrec]).

    For leap-frog the returned U is (u^n, v unchanged, w_x^n, w_y^n).
    """
    U = model.zeros_state() if U0 is None else tuple(f.copy() for f in U0)
    seis = [] if rec_nodes is not None else None
    if method == "faber" and faber_params is None:
        faber_params = ellipse_params(model.c_max, model.beta0, model.dx, model.order,
                                      free_surface=model.free_surface)
    if method == "leapfrog":
        LF = leapfrog_init(U)
    for n in range(nsteps):
        t_n = t0 + n * dt
        if method == "faber":
            U = faber_step(model, U, src, t_n, dt, m, faber_params)
        elif method == "krylov":
            U = krylov_step(model, U, src, t_n, dt, m)
        elif method == "hork":
            U = hork_step(model, U, src, t_n, dt, m)
        elif method == "rk32":
            U = rk32_step(model, U, src, t_n, dt)
        elif method == "rk44":
            U = rk44_step(model, U, src, t_n, dt)
        elif method == "leapfrog":
            LF = leapfrog_step(model, LF, src, t_n, dt, lf_variant)
            U = (LF[0], U[1], LF[2], LF[4])
        else:
            raise ValueError(method)
        if seis is not None:
            seis.append(record(U[0], rec_nodes))
    S = np.array(seis) if seis is not None else None
    return U, S

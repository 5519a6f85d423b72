"""Leap-frog two-step scheme of the oracle (Sec. 3.1, "Two step method").

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 3.1 solves u_tt = -bx by u - (bx + by) u_t + c^2 (u_xx + u_yy + d_x w_x + d_y w_y) + f and
w_{z,t} = -bz w_z + (b' - bz) d_z u with u_tt ~ (u^{n+1} - 2u^n + u^{n-1})/dt^2 and
w_t ~ (w^{n+1} - w^{n-1})/(2 dt).  Readings of what Sec. 3.1 leaves open:

* u_t in the damping term is the centred (u^{n+1} - u^{n-1})/(2 dt), solved pointwise:
  u^{n+1} (1/dt^2 + b/(2dt)) = (2u^n - u^{n-1})/dt^2 + b u^{n-1}/(2dt) - bx by u^n
  + c^2 (L u^n + d_x w_x^n + d_y w_y^n) + f(t_n).
* ``variant="averaged"`` (default): the damping of w is time-averaged,
  -bz (w^{n+1} + w^{n-1})/2, so (1 + bz dt) w^{n+1} = (1 - bz dt) w^{n-1} + 2 dt (b' - bz) d_z u^n.
  ``variant="literal"``: -bz w^n explicit, w^{n+1} = w^{n-1} + 2 dt (-bz w^n + (b' - bz) d_z u^n)
  (it has a parasitic mode with |zeta| = bz dt + sqrt(1 + bz^2 dt^2) > 1 inside the PML).
* Start: u^{-1} = u^0 and w^{-1} = w^0 (zero initial fields in all experiments).

The state is (u^n, u^{n-1}, w_x^n, w_x^{n-1}, w_y^n, w_y^{n-1}).

Pins: tests/test_oracle_integrators.py (second-order convergence; conservation of the
discrete leap-frog energy at beta = 0 without free surface).
"""
import numpy as np

from .operator import dx_half, dx_node, dxx, dy_half, dy_node, dyy


def leapfrog_init(U):
    u, _v, wx, wy = U
    return (u.copy(), u.copy(), wx.copy(), wx.copy(), wy.copy(), wy.copy())


def leapfrog_step(model, LF, src, t_n, dt, variant="averaged"):
    u, um, wx, wxm, wy, wym = LF
    bxn = model.beta_x_node()[None, :]
    byn = model.beta_y_node()[:, None]
    bxh = model.beta_x_half()[None, :]
    byh = model.beta_y_half()[:, None]
    b = bxn + byn
    rhs = (-bxn * byn * u + model.c2 * (dxx(model, u) + dyy(model, u)
                                        + dx_node(model, wx) + dy_node(model, wy)))
    if src is not None:
        rhs[src.j, src.i] += src.f(t_n)
    up = ((2.0 * u - um) / dt ** 2 + b * um / (2.0 * dt) + rhs) / (1.0 / dt ** 2 + b / (2.0 * dt))
    gx = (byn - bxh) * dx_half(model, u)
    gy = (bxn - byh) * dy_half(model, u)
    if variant == "averaged":
        wxp = ((1.0 - bxh * dt) * wxm + 2.0 * dt * gx) / (1.0 + bxh * dt)
        wyp = ((1.0 - byh * dt) * wym + 2.0 * dt * gy) / (1.0 + byh * dt)
    elif variant == "literal":
        wxp = wxm + 2.0 * dt * (-bxh * wx + gx)
        wyp = wym + 2.0 * dt * (-byh * wy + gy)
    else:
        raise ValueError("variant must be 'averaged' or 'literal'")
    return (up, u, wxp, wx, wyp, wy)

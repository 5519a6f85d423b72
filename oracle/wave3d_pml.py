"""Three-dimensional PML with an auxiliary field (oracle; groundwork for a 3D path whose
absorbing layer reduces exactly to Eq. 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper is two-dimensional.  Its Eq. 1 is the auxiliary-field form of the PML wave equation
u_tt + (b_x + b_y) u_t + b_x b_y u = c^2 (lap u + div w).  In three dimensions the same
complex-coordinate stretching (s_a = 1 + b_a / (i omega) on each axis) leaves a term
b_x b_y b_z times the time integral of u, carried here by psi, psi_t = u (the published
auxiliary-field PML for the second-order wave equation has this structure).  State
U = (u, v, w_x, w_y, w_z, psi):

    (HU)_u   = v
    (HU)_v   = -(b_x b_y + b_y b_z + b_x b_z) u - (b_x + b_y + b_z) v - b_x b_y b_z psi
               + c^2 (lap u + d_x w_x + d_y w_y + d_z w_z)            (+ source)
    (HU)_w_a = (sum of the other two b's - b_a) d_a u + (product of the other two b's) d_a psi
               - b_a w_a,                                              a = x, y, z
    (HU)_psi = u

Placement, stencils, free-surface rows and damping profile are those of ``oracle.wave3d``:
in a w_a row b_a is taken at the half point and the other two at the nodes; psi lives at the
nodes and d_a psi uses the same half-point stencil as d_a u.  With one axis undamped and a
field that does not vary along it, the u, v and remaining w rows are exactly Eq. 1 on the
other two axes (the product terms vanish), which ``oracle.wave3d``'s mean-of-the-others
reading does not achieve.  ``undamped`` names axes whose damping is switched off (for that
pin).

Two routes: ``apply_H3p`` (shifted arrays, reusing the derivative operators of
``oracle.wave3d``) and ``assemble_H3p`` (tap-by-tap sparse assembly written out here).

Leap-frog (Sec. 3.1's two-step scheme) on this PML, ``leapfrog3dp_step``: u and the w fields
as in ``oracle.wave3d.leapfrog3d_step`` (u_t of the damping term centred, the damping of w
time-averaged) with the psi terms added at level n, and psi advanced by the trapezoid rule,
psi^{n+1} = psi^n + dt (u^n + u^{n+1}) / 2 (the paper is 2D and has no psi: this is the
reading of its scheme for the extra field).
``Model3DPML`` is a ``Model3D`` whose state carries psi; ``oracle.operator.apply_H`` sends it
to ``apply_H3p``, so every integrator of the oracle runs on this PML.
Pins: tests/test_oracle_wave3d_pml.py (also: the integrators against the dense exponential,
and a pulse absorbed over 10x better than with ``oracle.wave3d``'s layer).
"""
import numpy as np
import scipy.sparse as sp

from . import stencils as S
from . import wave3d as W
from .wave3d import d_half, d_node, d_second


def _profiles(m, undamped=()):
    """Node and half-point damping of the three axes, with the ``undamped`` ones zeroed."""
    prof = {"x": (m.beta_x(), m.beta_x(True)), "y": (m.beta_y(), m.beta_y(True)),
            "z": (m.beta_z(), m.beta_z(True))}
    return {a: ((0 * n, 0 * h) if a in undamped else (n, h)) for a, (n, h) in prof.items()}


def field_shapes(m):
    """Shapes of (u, v, w_x, w_y, w_z, psi) on a ``Model3D`` grid."""
    return list(W.Model3D.field_shapes(m)) + [(m.nz, m.ny, m.nx)]


class Model3DPML(W.Model3D):
    """A ``Model3D`` whose operator is ``apply_H3p``: its state carries psi, so every integrator
    of the oracle (which reaches H through ``oracle.operator.apply_H``) runs on this PML."""

    aux_psi = True

    def field_shapes(self):
        return field_shapes(self)


def apply_H3p(m, state, src=None, undamped=()):
    """H U of the module header; ``src`` is None or (k, j, i, value) added to the v row."""
    u, v, wx, wy, wz, psi = state
    p = _profiles(m, undamped)
    bx, bxh = p["x"][0][None, None, :], p["x"][1][None, None, :]
    by, byh = p["y"][0][None, :, None], p["y"][1][None, :, None]
    bz, bzh = p["z"][0][:, None, None], p["z"][1][:, None, None]
    lap = d_second(m, u, 2) + d_second(m, u, 1) + d_second(m, u, 0)
    div = d_node(m, wx, 2) + d_node(m, wy, 1) + d_node(m, wz, 0)
    hv = (-(bx * by + by * bz + bx * bz) * u - (bx + by + bz) * v - bx * by * bz * psi
          + m.c2 * (lap + div))
    hwx = (by + bz - bxh) * d_half(m, u, 2) + by * bz * d_half(m, psi, 2) - bxh * wx
    hwy = (bx + bz - byh) * d_half(m, u, 1) + bx * bz * d_half(m, psi, 1) - byh * wy
    hwz = (bx + by - bzh) * d_half(m, u, 0) + bx * by * d_half(m, psi, 0) - bzh * wz
    if src is not None:
        k, j, i, val = src
        hv = hv.copy()
        hv[k, j, i] += val
    return (v.copy(), hv, hwx, hwy, hwz, u.copy())


def assemble_H3p(m, undamped=()):
    """Sparse H (CSR) of ``apply_H3p``, one stencil tap at a time (taps off the grid dropped)."""
    nx, ny, nz, dx = m.nx, m.ny, m.nz, m.dx
    R = S.half_width(m.order)
    s = [float(c) for c in S.STAG[m.order]]
    d = [float(c) for c in S.CENT[m.order]]
    fs = m.free_surface
    fs_uzz, fs_uz, fs_dwz = S.as_float(S.FS_UYY), S.as_float(S.FS_UY), S.as_float(S.FS_DWY)
    N = nx * ny * nz
    o_wx = 2 * N
    o_wy = o_wx + nz * ny * (nx - 1)
    o_wz = o_wy + nz * (ny - 1) * nx
    o_psi = o_wz + (nz - 1) * ny * nx
    p = _profiles(m, undamped)
    bx, bxh = p["x"]
    by, byh = p["y"]
    bz, bzh = p["z"]
    c2 = m.c2
    rows, cols, vals = [], [], []

    def put(r, c, w):
        rows.append(r)
        cols.append(c)
        vals.append(w)

    def U(k, j, i):
        return (k * ny + j) * nx + i

    def PSI(k, j, i):
        return o_psi + U(k, j, i)

    def WX(k, j, i):
        return o_wx + (k * ny + j) * (nx - 1) + i

    def WY(k, j, i):
        return o_wy + (k * (ny - 1) + j) * nx + i

    def WZ(k, j, i):
        return o_wz + (k * ny + j) * nx + i

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                put(U(k, j, i), N + U(k, j, i), 1.0)               # u row
                put(PSI(k, j, i), U(k, j, i), 1.0)                 # psi row
                r = N + U(k, j, i)                                 # v row
                put(r, U(k, j, i), -(bx[i] * by[j] + by[j] * bz[k] + bx[i] * bz[k]))
                put(r, r, -(bx[i] + by[j] + bz[k]))
                put(r, PSI(k, j, i), -bx[i] * by[j] * bz[k])
                k2, k1 = c2[k, j, i] / (dx * dx), c2[k, j, i] / dx
                for off in range(-R, R + 1):
                    if 0 <= i + off < nx:
                        put(r, U(k, j, i + off), k2 * d[abs(off)])
                    if 0 <= j + off < ny:
                        put(r, U(k, j + off, i), k2 * d[abs(off)])
                if fs and k < S.N_FS_UYY_ROWS:
                    for q in range(fs_uzz.shape[1]):
                        if q < nz:
                            put(r, U(q, j, i), k2 * fs_uzz[k, q])
                else:
                    for off in range(-R, R + 1):
                        if 0 <= k + off < nz:
                            put(r, U(k + off, j, i), k2 * d[abs(off)])
                for q in range(R):
                    if 0 <= i + q < nx - 1:
                        put(r, WX(k, j, i + q), k1 * s[q])
                    if 0 <= i - 1 - q < nx - 1:
                        put(r, WX(k, j, i - 1 - q), -k1 * s[q])
                    if 0 <= j + q < ny - 1:
                        put(r, WY(k, j + q, i), k1 * s[q])
                    if 0 <= j - 1 - q < ny - 1:
                        put(r, WY(k, j - 1 - q, i), -k1 * s[q])
                if fs and k < S.N_FS_UYY_ROWS:
                    for q in range(fs_dwz.shape[1]):
                        if q < nz - 1:
                            put(r, WZ(q, j, i), k1 * fs_dwz[k, q])
                else:
                    for q in range(R):
                        if 0 <= k - 1 - q < nz - 1:
                            put(r, WZ(k - 1 - q, j, i), k1 * s[q])
                        if 0 <= k + q < nz - 1:
                            put(r, WZ(k + q, j, i), -k1 * s[q])
    # w rows: (sum of the other b's - b_a) d_a u + (product of the other b's) d_a psi - b_a w_a
    for k in range(nz):
        for j in range(ny):
            for i in range(nx - 1):
                r = WX(k, j, i)
                put(r, r, -bxh[i])
                gu = (by[j] + bz[k] - bxh[i]) / dx
                gp = by[j] * bz[k] / dx
                for q in range(R):
                    if i + 1 + q < nx:
                        put(r, U(k, j, i + 1 + q), gu * s[q])
                        put(r, PSI(k, j, i + 1 + q), gp * s[q])
                    if i - q >= 0:
                        put(r, U(k, j, i - q), -gu * s[q])
                        put(r, PSI(k, j, i - q), -gp * s[q])
    for k in range(nz):
        for j in range(ny - 1):
            for i in range(nx):
                r = WY(k, j, i)
                put(r, r, -byh[j])
                gu = (bx[i] + bz[k] - byh[j]) / dx
                gp = bx[i] * bz[k] / dx
                for q in range(R):
                    if j + 1 + q < ny:
                        put(r, U(k, j + 1 + q, i), gu * s[q])
                        put(r, PSI(k, j + 1 + q, i), gp * s[q])
                    if j - q >= 0:
                        put(r, U(k, j - q, i), -gu * s[q])
                        put(r, PSI(k, j - q, i), -gp * s[q])
    for k in range(nz - 1):
        for j in range(ny):
            for i in range(nx):
                r = WZ(k, j, i)
                put(r, r, -bzh[k])
                gu = (bx[i] + by[j] - bzh[k]) / dx
                gp = bx[i] * by[j] / dx
                if fs and k < S.N_FS_UY_ROWS:
                    for q in range(fs_uz.shape[1]):
                        if q < nz:
                            put(r, U(q, j, i), gu * fs_uz[k, q])
                            put(r, PSI(q, j, i), gp * fs_uz[k, q])
                else:
                    for q in range(R):          # upward: u_{k-q} - u_{k+1+q}
                        if k - q >= 0:
                            put(r, U(k - q, j, i), gu * s[q])
                            put(r, PSI(k - q, j, i), gp * s[q])
                        if k + 1 + q < nz:
                            put(r, U(k + 1 + q, j, i), -gu * s[q])
                            put(r, PSI(k + 1 + q, j, i), -gp * s[q])
    n = o_psi + N
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


# ------------------------------------------------------------------ leap-frog
def leapfrog3dp_init(U):
    """Leap-frog state (u^n, u^{n-1}, w_x^n, w_x^{n-1}, w_y^n, w_y^{n-1}, w_z^n, w_z^{n-1},
    psi^n) from U = (u, v, w_x, w_y, w_z, psi) with u^{-1} = u^0 and w^{-1} = w^0."""
    u, _v, wx, wy, wz, psi = U
    return (u.copy(), u.copy(), wx.copy(), wx.copy(), wy.copy(), wy.copy(), wz.copy(), wz.copy(),
            psi.copy())


def leapfrog3dp_step(m, LF, src, t_n, dt, undamped=()):
    """One step of the scheme in the module header."""
    u, um, wx, wxm, wy, wym, wz, wzm, psi = LF
    p = _profiles(m, undamped)
    bx, bxh = p["x"][0][None, None, :], p["x"][1][None, None, :]
    by, byh = p["y"][0][None, :, None], p["y"][1][None, :, None]
    bz, bzh = p["z"][0][:, None, None], p["z"][1][:, None, None]
    b = bx + by + bz
    lap = d_second(m, u, 2) + d_second(m, u, 1) + d_second(m, u, 0)
    div = d_node(m, wx, 2) + d_node(m, wy, 1) + d_node(m, wz, 0)
    rhs = -(bx * by + by * bz + bx * bz) * u - bx * by * bz * psi + m.c2 * (lap + div)
    if src is not None:
        rhs[src.k, src.j, src.i] += src.f(t_n)
    up = ((2.0 * u - um) / dt ** 2 + b * um / (2.0 * dt) + rhs) / (1.0 / dt ** 2 + b / (2.0 * dt))

    def wnext(wm, bh, g):
        return ((1.0 - bh * dt) * wm + 2.0 * dt * g) / (1.0 + bh * dt)

    wxp = wnext(wxm, bxh, (by + bz - bxh) * d_half(m, u, 2) + by * bz * d_half(m, psi, 2))
    wyp = wnext(wym, byh, (bx + bz - byh) * d_half(m, u, 1) + bx * bz * d_half(m, psi, 1))
    wzp = wnext(wzm, bzh, (bx + by - bzh) * d_half(m, u, 0) + bx * by * d_half(m, psi, 0))
    psip = psi + 0.5 * dt * (u + up)
    return (up, u, wxp, wx, wyp, wy, wzp, wz, psip)

"""The semi-discrete operator H of Eq. (1), matrix-free and as an assembled sparse matrix.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Eq. (1) (Sec. 2), applied to U = (u, v, w_x, w_y):

    (HU)_u   = v
    (HU)_v   = -bx by u + c^2 (u_xx + u_yy) - (bx + by) v + c^2 (d_x w_x + d_y w_y)
    (HU)_w_x = (by - bx) d_x u - bx w_x            at (i+1/2, j)
    (HU)_w_y = (bx - by) d_y u - by w_y            at (i, j+1/2)

with the stencils of ``oracle.stencils``: interior 8th-order (or 4th-order) staggered first
derivatives and centred second derivatives (Sec. 2.1), zero extension beyond the grid on
the sides and bottom (and top without free surface), and, with a free surface (Sec. 2.2 and
Appendix A), one-sided u_yy rows at j = 0..3, u_y rows at half rows 0..2 and Fornberg rows
for d_y w_y at j = 0..3.  y is the paper's upward coordinate: the row index j grows
downward, so an interior d_y at half row j+1/2 is sum_k s_k (u_{j-k} - u_{j+1+k}) / dx.

Two independent routes:
* ``apply_H`` -- shifted-array (matrix-free) evaluation; the one the integrators use.
* ``assemble_H`` -- COO assembly of the same rows, one stencil tap at a time; its transpose
  gives H^T for the adjoint identity and for the oracle's adjoint integrators.

Pins: tests/test_oracle_operator.py (polynomial exactness and convergence order against
analytic derivatives, energy conservation at beta = 0, the two routes against each other).
"""
import numpy as np
import scipy.sparse as sp

from . import stencils as S
from .model import Model


def _coef(order):
    R = S.half_width(order)
    return R, S.as_float(S.STAG[order]), S.as_float(S.CENT[order])


def _pad(a, axis, lo, hi):
    pw = [(0, 0)] * a.ndim
    pw[axis] = (lo, hi)
    return np.pad(a, pw)


# ------------------------------------------------------------------ x derivatives
def dx_half(m, u):
    """d_x u at (i+1/2, j), i = 0..nx-2.  Eq. (spatial_8th_1)."""
    R, s, _ = _coef(m.order)
    nx = m.nx
    up = _pad(u, 1, R, R)              # up[:, R+q] = u[:, q]
    out = np.zeros((u.shape[0], nx - 1))
    for k in range(R):
        out += s[k] * (up[:, R + 1 + k:R + 1 + k + nx - 1] - up[:, R - k:R - k + nx - 1])
    return out / m.dx


def dx_node(m, wx):
    """d_x w_x at nodes (i, j), i = 0..nx-1; w_x[i] sits at i+1/2."""
    R, s, _ = _coef(m.order)
    nx = m.nx
    wp = _pad(wx, 1, R, R + 1)         # wp[:, R+q] = wx[:, q]
    out = np.zeros((wx.shape[0], nx))
    for k in range(R):
        out += s[k] * (wp[:, R + k:R + k + nx] - wp[:, R - 1 - k:R - 1 - k + nx])
    return out / m.dx


def dxx(m, u):
    """u_xx at nodes.  Eq. (spatial_8th_2) read with "+" between pairs."""
    R, _, d = _coef(m.order)
    nx = m.nx
    up = _pad(u, 1, R, R)
    out = d[0] * u
    for k in range(1, R + 1):
        out = out + d[k] * (up[:, R + k:R + k + nx] + up[:, R - k:R - k + nx])
    return out / (m.dx * m.dx)


# ------------------------------------------------------------------ y derivatives
def dy_half(m, u):
    """d_y u at (i, j+1/2), j = 0..ny-2, physical (upward) y."""
    R, s, _ = _coef(m.order)
    ny = m.ny
    up = _pad(u, 0, R, R)              # up[R+q] = u[q]
    out = np.zeros((ny - 1, u.shape[1]))
    for k in range(R):
        out += s[k] * (up[R - k:R - k + ny - 1] - up[R + 1 + k:R + 1 + k + ny - 1])
    if m.free_surface:
        fs = S.as_float(S.FS_UY)
        for j in range(min(S.N_FS_UY_ROWS, ny - 1)):
            row = np.zeros(u.shape[1])
            for q in range(fs.shape[1]):
                if q < ny:
                    row += fs[j, q] * u[q]
            out[j] = row
    return out / m.dx


def dy_node(m, wy):
    """d_y w_y at nodes (i, j); w_y[j] sits at j+1/2 (physical y)."""
    R, s, _ = _coef(m.order)
    ny = m.ny
    wp = _pad(wy, 0, R, R + 1)         # wp[R+q] = wy[q]
    out = np.zeros((ny, wy.shape[1]))
    for k in range(R):
        out += s[k] * (wp[R - 1 - k:R - 1 - k + ny] - wp[R + k:R + k + ny])
    if m.free_surface:
        fs = S.as_float(S.FS_DWY)
        for j in range(min(S.N_FS_UYY_ROWS, ny)):
            row = np.zeros(wy.shape[1])
            for q in range(fs.shape[1]):
                if q < ny - 1:
                    row += fs[j, q] * wy[q]
            out[j] = row
    return out / m.dx


def dyy(m, u):
    """u_yy at nodes; free-surface rows j = 0..3 from Appendix A."""
    R, _, d = _coef(m.order)
    ny = m.ny
    up = _pad(u, 0, R, R)
    out = d[0] * u
    for k in range(1, R + 1):
        out = out + d[k] * (up[R + k:R + k + ny] + up[R - k:R - k + ny])
    if m.free_surface:
        fs = S.as_float(S.FS_UYY)
        for j in range(min(S.N_FS_UYY_ROWS, ny)):
            row = np.zeros(u.shape[1])
            for q in range(fs.shape[1]):
                if q < ny:
                    row += fs[j, q] * u[q]
            out[j] = row
    return out / (m.dx * m.dx)


# ------------------------------------------------------------------ operator
def apply_H(m: Model, state, src=None):
    """H U (Eq. 1) plus an optional point source term.

    ``src`` is ``None`` or ``(j, i, value)``: ``value`` is added to the v-row at node (i, j)
    (the f entry of Eq. 1 / the W y term of the augmented matrix).  A three-dimensional
    model goes to ``oracle.wave3d.apply_H3`` (src ``(k, j, i, value)``), and one with the
    auxiliary field psi (``oracle.wave3d_pml.Model3DPML``) to ``apply_H3p``.
    """
    if getattr(m, "aux_psi", False):
        from .wave3d_pml import apply_H3p
        return apply_H3p(m, state, src)
    if getattr(m, "dims", 2) == 3:
        from .wave3d import apply_H3
        return apply_H3(m, state, src)
    u, v, wx, wy = state
    bxn = m.beta_x_node()[None, :]
    byn = m.beta_y_node()[:, None]
    bxh = m.beta_x_half()[None, :]
    byh = m.beta_y_half()[:, None]
    c2 = m.c2
    hu = v.copy()
    hv = (-bxn * byn * u + c2 * (dxx(m, u) + dyy(m, u)) - (bxn + byn) * v
          + c2 * (dx_node(m, wx) + dy_node(m, wy)))
    hwx = (byn - bxh) * dx_half(m, u) - bxh * wx
    hwy = (bxn - byh) * dy_half(m, u) - byh * wy
    if src is not None:
        j, i, val = src
        hv[j, i] += val
    return (hu, hv, hwx, hwy)


# ------------------------------------------------------------------ sparse assembly
class _Index:
    """Flat indices of (u, v, w_x, w_y) in the ``flatten`` order."""

    def __init__(self, m):
        nx, ny = m.nx, m.ny
        self.nx, self.ny = nx, ny
        self.ou = 0
        self.ov = nx * ny
        self.owx = 2 * nx * ny
        self.owy = 2 * nx * ny + (nx - 1) * ny

    def u(self, j, i):
        return self.ou + j * self.nx + i

    def v(self, j, i):
        return self.ov + j * self.nx + i

    def wx(self, j, i):
        return self.owx + j * (self.nx - 1) + i

    def wy(self, j, i):
        return self.owy + j * self.nx + i


def assemble_H(m: Model):
    """Sparse H (CSR), built row by row from the stencil tables (independent of apply_H).

    Each row of Eq. (1) is written as a list of (column, weight) taps; taps that fall
    outside the grid are dropped (zero extension).
    """
    nx, ny, dx = m.nx, m.ny, m.dx
    R = S.half_width(m.order)
    s = [float(c) for c in S.STAG[m.order]]
    d = [float(c) for c in S.CENT[m.order]]
    fs_uyy = S.as_float(S.FS_UYY) if m.free_surface else None
    fs_uy = S.as_float(S.FS_UY) if m.free_surface else None
    fs_dwy = S.as_float(S.FS_DWY) if m.free_surface else None
    ix = _Index(m)
    bxn, byn = m.beta_x_node(), m.beta_y_node()
    bxh, byh = m.beta_x_half(), m.beta_y_half()
    c2 = m.c2
    rows, cols, vals = [], [], []

    def put(r, c, w):
        rows.append(r)
        cols.append(c)
        vals.append(w)

    for j in range(ny):
        for i in range(nx):
            # u-row: u_t = v
            put(ix.u(j, i), ix.v(j, i), 1.0)
            # v-row
            r = ix.v(j, i)
            put(r, ix.u(j, i), -bxn[i] * byn[j])
            put(r, ix.v(j, i), -(bxn[i] + byn[j]))
            k2 = c2[j, i] / (dx * dx)
            # u_xx
            for off in range(-R, R + 1):
                if 0 <= i + off < nx:
                    put(r, ix.u(j, i + off), k2 * d[abs(off)])
            # u_yy
            if m.free_surface and j < S.N_FS_UYY_ROWS:
                for q in range(fs_uyy.shape[1]):
                    if q < ny:
                        put(r, ix.u(q, i), k2 * fs_uyy[j, q])
            else:
                for off in range(-R, R + 1):
                    if 0 <= j + off < ny:
                        put(r, ix.u(j + off, i), k2 * d[abs(off)])
            k1 = c2[j, i] / dx
            # d_x w_x at node i: w_x[i+k] (+), w_x[i-1-k] (-)
            for k in range(R):
                if 0 <= i + k < nx - 1:
                    put(r, ix.wx(j, i + k), k1 * s[k])
                if 0 <= i - 1 - k < nx - 1:
                    put(r, ix.wx(j, i - 1 - k), -k1 * s[k])
            # d_y w_y at node j: w_y[j-1-k] (+), w_y[j+k] (-)
            if m.free_surface and j < S.N_FS_UYY_ROWS:
                for q in range(fs_dwy.shape[1]):
                    if q < ny - 1:
                        put(r, ix.wy(q, i), k1 * fs_dwy[j, q])
            else:
                for k in range(R):
                    if 0 <= j - 1 - k < ny - 1:
                        put(r, ix.wy(j - 1 - k, i), k1 * s[k])
                    if 0 <= j + k < ny - 1:
                        put(r, ix.wy(j + k, i), -k1 * s[k])
    # w_x rows
    for j in range(ny):
        for i in range(nx - 1):
            r = ix.wx(j, i)
            put(r, r, -bxh[i])
            g = (byn[j] - bxh[i]) / dx
            for k in range(R):
                if 0 <= i + 1 + k < nx:
                    put(r, ix.u(j, i + 1 + k), g * s[k])
                if 0 <= i - k < nx:
                    put(r, ix.u(j, i - k), -g * s[k])
    # w_y rows
    for j in range(ny - 1):
        for i in range(nx):
            r = ix.wy(j, i)
            put(r, r, -byh[j])
            g = (bxn[i] - byh[j]) / dx
            if m.free_surface and j < S.N_FS_UY_ROWS:
                for q in range(fs_uy.shape[1]):
                    if q < ny:
                        put(r, ix.u(q, i), g * fs_uy[j, q])
            else:
                for k in range(R):
                    if 0 <= j - k < ny:
                        put(r, ix.u(j - k, i), g * s[k])
                    if 0 <= j + 1 + k < ny:
                        put(r, ix.u(j + 1 + k, i), -g * s[k])
    n = m.n
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))

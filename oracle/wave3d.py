"""Three-dimensional extension of the PML operator, for the 400^3 throughput workload (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper is two-dimensional (Eq. 1, Sec. 2).  This module is the builder's own extension.
Without damping it reduces to Eq. 1 when one axis is dropped, and with one axis undamped its
v row does too; its w rows use the mean of the other two damping profiles, so with damping
they do not (a PML that reduces exactly needs a further auxiliary field).  The damping is
this extension's own reading.  State U = (u, v, w_x, w_y, w_z);
x, y horizontal (i, j), z vertical (k = 0 the top, depth grows with k):

    (HU)_u   = v
    (HU)_v   = -(bx by + by bz + bx bz) u - (bx + by + bz) v
               + c^2 (u_xx + u_yy + u_zz + d_x w_x + d_y w_y + d_z w_z)  (+ source)
    (HU)_w_a = (mean of the other two b's - b_a) d_a u - b_a w_a,   a = x, y, z

with w_x at (i+1/2, j, k), w_y at (i, j+1/2, k) and w_z at (i, j, k+1/2).  In each w_a row, b_a
is taken at the half point and the other two b's at the nodes; the v row takes all three at the
node.  The stencils are those of Sec. 2.1.  Zero extension applies beyond the grid.  The
damping profile is Sec. 2's beta0 (1 - d/delta)^2, with the boundary on the ghost line, as in
``oracle.model``.  With a free surface at k = 0, the z axis plays the part of the 2D y axis:

* z points upward, so d_z at half level k+1/2 is sum_q s_q (u_{k-q} - u_{k+1+q}) / dx;
* Appendix A's one-sided rows replace u_zz at k = 0..3 and d_z u at half levels 0..2;
* the Fornberg rows replace d_z w_z at k = 0..3;
* the top strip has no z damping.

Two routes, as in 2D: ``apply_H3`` (shifted arrays) and ``assemble_H3`` (tap-by-tap sparse
assembly, whose transpose serves the adjoint identity).

Pins (tests/test_oracle_wave3d.py):
* the two routes agree;
* polynomial exactness of every derivative away from the boundary;
* at beta = 0 and without a free surface, the Laplacian block is symmetric;
* at beta = 0, a field constant in y gives, on the interior y rows, exactly the 2D operator of
  ``oracle.operator`` on the x-z slice (free-surface rows included);
* every integrator converges to the dense exponential on a tiny grid.

The damping coefficients of the w rows are this extension's own choice: "parity unpinned"
beyond the consistency checks above.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import stencils as S
from .source import PointSource, node_index


@dataclass
class Model3D:
    nx: int
    ny: int
    nz: int
    dx: float
    order: int
    pml: int
    beta0: float
    free_surface: bool
    c: np.ndarray = field(repr=False)   # velocity at nodes, shape (nz, ny, nx)

    dims = 3

    def __post_init__(self):
        self.c = np.asarray(self.c, dtype=np.float64)
        if self.c.shape != (self.nz, self.ny, self.nx):
            raise ValueError("c must have shape (nz, ny, nx)")
        if self.order not in (4, 8):
            raise ValueError("order must be 4 or 8")
        if self.free_surface and self.order != 8:
            raise ValueError("free-surface rows exist for 8th order only")
        if min(self.nx, self.ny, self.nz) < 2:
            raise ValueError("grid must be at least 2 x 2 x 2")

    @property
    def c2(self):
        return self.c * self.c

    @property
    def c_max(self):
        return float(self.c.max())

    # -- damping --------------------------------------------------------------------
    def _beta(self, d):
        d = np.asarray(d, dtype=np.float64)
        if self.pml <= 0:
            return np.zeros_like(d)
        return np.where(d <= self.pml, self.beta0 * (1.0 - d / self.pml) ** 2, 0.0)

    def _two_sided(self, n, half):
        i = np.arange(n - 1 if half else n, dtype=np.float64)
        return self._beta(np.minimum(i + 1.5, n - i - 0.5) if half else np.minimum(i + 1.0, n - i))

    def beta_x(self, half=False):
        return self._two_sided(self.nx, half)

    def beta_y(self, half=False):
        return self._two_sided(self.ny, half)

    def beta_z(self, half=False):
        if not self.free_surface:
            return self._two_sided(self.nz, half)
        k = np.arange(self.nz - 1 if half else self.nz, dtype=np.float64)
        return self._beta(self.nz - k - 0.5 if half else self.nz - k)

    # -- sizes ----------------------------------------------------------------------
    def field_shapes(self):
        nx, ny, nz = self.nx, self.ny, self.nz
        return [(nz, ny, nx), (nz, ny, nx), (nz, ny, nx - 1), (nz, ny - 1, nx), (nz - 1, ny, nx)]

    @property
    def n(self):
        return sum(int(np.prod(s)) for s in self.field_shapes())

    def zeros_state(self):
        return tuple(np.zeros(s) for s in self.field_shapes())


# ------------------------------------------------------------------ derivatives
def _coef(order):
    return S.half_width(order), S.as_float(S.STAG[order]), S.as_float(S.CENT[order])


def _shift(a, axis, off, n_out):
    """Slice a[off : off + n_out] along ``axis`` of the zero-extended array (any off)."""
    n = a.shape[axis]
    lo, hi = off, off + n_out
    pad_lo, pad_hi = max(0, -lo), max(0, hi - n)
    pw = [(0, 0)] * a.ndim
    pw[axis] = (pad_lo, pad_hi)
    ap = np.pad(a, pw)
    sl = [slice(None)] * a.ndim
    sl[axis] = slice(lo + pad_lo, hi + pad_lo)
    return ap[tuple(sl)]


def d_half(m, u, axis):
    """d_a u at the half points along ``axis`` (x: 2, y: 1 rightward; z: 0 upward with the
    free-surface half rows 0..2)."""
    R, s, _ = _coef(m.order)
    n = u.shape[axis]
    out = 0.0
    for q in range(R):
        out = out + s[q] * (_shift(u, axis, 1 + q, n - 1) - _shift(u, axis, -q, n - 1))
    if axis == 0:
        out = -out
        if m.free_surface:
            fs = S.as_float(S.FS_UY)
            out = np.array(out)
            for k in range(min(S.N_FS_UY_ROWS, n - 1)):
                out[k] = sum(fs[k, q] * u[q] for q in range(fs.shape[1]) if q < n)
    return out / m.dx


def d_node(m, w, axis):
    """d_a w_a at the nodes from w_a on the half points along ``axis``."""
    R, s, _ = _coef(m.order)
    n = w.shape[axis] + 1
    out = 0.0
    for q in range(R):
        out = out + s[q] * (_shift(w, axis, q, n) - _shift(w, axis, -1 - q, n))
    if axis == 0:
        out = -out
        if m.free_surface:
            fs = S.as_float(S.FS_DWY)
            out = np.array(out)
            for k in range(min(S.N_FS_UYY_ROWS, n)):
                out[k] = sum(fs[k, q] * w[q] for q in range(fs.shape[1]) if q < n - 1)
    return out / m.dx


def d_second(m, u, axis):
    """u_aa at the nodes (centred; Appendix A rows 0..3 on z with a free surface)."""
    R, _, d = _coef(m.order)
    n = u.shape[axis]
    out = d[0] * u
    for q in range(1, R + 1):
        out = out + d[q] * (_shift(u, axis, q, n) + _shift(u, axis, -q, n))
    if axis == 0 and m.free_surface:
        fs = S.as_float(S.FS_UYY)
        out = np.array(out)
        for k in range(min(S.N_FS_UYY_ROWS, n)):
            out[k] = sum(fs[k, q] * u[q] for q in range(fs.shape[1]) if q < n)
    return out / (m.dx * m.dx)


def _betas(m):
    bx, by, bz = m.beta_x(), m.beta_y(), m.beta_z()
    return bx[None, None, :], by[None, :, None], bz[:, None, None]


def apply_H3(m, state, src=None):
    """H U of the module header; ``src`` is None or (k, j, i, value) added to the v row."""
    u, v, wx, wy, wz = state
    bx, by, bz = _betas(m)
    bxh = m.beta_x(True)[None, None, :]
    byh = m.beta_y(True)[None, :, None]
    bzh = m.beta_z(True)[:, None, None]
    c2 = m.c2
    lap = d_second(m, u, 2) + d_second(m, u, 1) + d_second(m, u, 0)
    div = d_node(m, wx, 2) + d_node(m, wy, 1) + d_node(m, wz, 0)
    hu = v.copy()
    hv = -(bx * by + by * bz + bx * bz) * u - (bx + by + bz) * v + c2 * (lap + div)
    hwx = (0.5 * (by + bz) - bxh) * d_half(m, u, 2) - bxh * wx
    hwy = (0.5 * (bx + bz) - byh) * d_half(m, u, 1) - byh * wy
    hwz = (0.5 * (bx + by) - bzh) * d_half(m, u, 0) - bzh * wz
    if src is not None:
        k, j, i, val = src
        hv[k, j, i] += val
    return (hu, hv, hwx, hwy, hwz)


# ------------------------------------------------------------------ sparse assembly
def assemble_H3(m):
    """Sparse H (CSR) of ``apply_H3``, one stencil tap at a time (taps off the grid dropped)."""
    nx, ny, nz, dx = m.nx, m.ny, m.nz, m.dx
    R = S.half_width(m.order)
    s = [float(c) for c in S.STAG[m.order]]
    d = [float(c) for c in S.CENT[m.order]]
    fs = m.free_surface
    fs_uzz = S.as_float(S.FS_UYY)
    fs_uz = S.as_float(S.FS_UY)
    fs_dwz = S.as_float(S.FS_DWY)
    N = nx * ny * nz
    o_wx = 2 * N
    o_wy = o_wx + nz * ny * (nx - 1)
    o_wz = o_wy + nz * (ny - 1) * nx

    def U(k, j, i):
        return (k * ny + j) * nx + i

    def V(k, j, i):
        return N + U(k, j, i)

    def WX(k, j, i):
        return o_wx + (k * ny + j) * (nx - 1) + i

    def WY(k, j, i):
        return o_wy + (k * (ny - 1) + j) * nx + i

    def WZ(k, j, i):
        return o_wz + (k * ny + j) * nx + i

    bx, by, bz = m.beta_x(), m.beta_y(), m.beta_z()
    bxh, byh, bzh = m.beta_x(True), m.beta_y(True), m.beta_z(True)
    c2 = m.c2
    rows, cols, vals = [], [], []

    def put(r, c, w):
        rows.append(r)
        cols.append(c)
        vals.append(w)

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                put(U(k, j, i), V(k, j, i), 1.0)
                r = V(k, j, i)
                put(r, U(k, j, i), -(bx[i] * by[j] + by[j] * bz[k] + bx[i] * bz[k]))
                put(r, V(k, j, i), -(bx[i] + by[j] + bz[k]))
                k2, k1 = c2[k, j, i] / (dx * dx), c2[k, j, i] / dx
                for off in range(-R, R + 1):          # u_xx, u_yy
                    if 0 <= i + off < nx:
                        put(r, U(k, j, i + off), k2 * d[abs(off)])
                    if 0 <= j + off < ny:
                        put(r, U(k, j + off, i), k2 * d[abs(off)])
                if fs and k < S.N_FS_UYY_ROWS:       # u_zz
                    for q in range(fs_uzz.shape[1]):
                        if q < nz:
                            put(r, U(q, j, i), k2 * fs_uzz[k, q])
                else:
                    for off in range(-R, R + 1):
                        if 0 <= k + off < nz:
                            put(r, U(k + off, j, i), k2 * d[abs(off)])
                for q in range(R):                    # d_x w_x, d_y w_y (rightward)
                    if 0 <= i + q < nx - 1:
                        put(r, WX(k, j, i + q), k1 * s[q])
                    if 0 <= i - 1 - q < nx - 1:
                        put(r, WX(k, j, i - 1 - q), -k1 * s[q])
                    if 0 <= j + q < ny - 1:
                        put(r, WY(k, j + q, i), k1 * s[q])
                    if 0 <= j - 1 - q < ny - 1:
                        put(r, WY(k, j - 1 - q, i), -k1 * s[q])
                if fs and k < S.N_FS_UYY_ROWS:       # d_z w_z (upward)
                    for q in range(fs_dwz.shape[1]):
                        if q < nz - 1:
                            put(r, WZ(q, j, i), k1 * fs_dwz[k, q])
                else:
                    for q in range(R):
                        if 0 <= k - 1 - q < nz - 1:
                            put(r, WZ(k - 1 - q, j, i), k1 * s[q])
                        if 0 <= k + q < nz - 1:
                            put(r, WZ(k + q, j, i), -k1 * s[q])
    for k in range(nz):
        for j in range(ny):
            for i in range(nx - 1):
                r = WX(k, j, i)
                put(r, r, -bxh[i])
                g = (0.5 * (by[j] + bz[k]) - bxh[i]) / dx
                for q in range(R):
                    if i + 1 + q < nx:
                        put(r, U(k, j, i + 1 + q), g * s[q])
                    if i - q >= 0:
                        put(r, U(k, j, i - q), -g * s[q])
    for k in range(nz):
        for j in range(ny - 1):
            for i in range(nx):
                r = WY(k, j, i)
                put(r, r, -byh[j])
                g = (0.5 * (bx[i] + bz[k]) - byh[j]) / dx
                for q in range(R):
                    if j + 1 + q < ny:
                        put(r, U(k, j + 1 + q, i), g * s[q])
                    if j - q >= 0:
                        put(r, U(k, j - q, i), -g * s[q])
    for k in range(nz - 1):
        for j in range(ny):
            for i in range(nx):
                r = WZ(k, j, i)
                put(r, r, -bzh[k])
                g = (0.5 * (bx[i] + by[j]) - bzh[k]) / dx
                if fs and k < S.N_FS_UY_ROWS:
                    for q in range(fs_uz.shape[1]):
                        if q < nz:
                            put(r, U(q, j, i), g * fs_uz[k, q])
                else:
                    for q in range(R):
                        if k - q >= 0:
                            put(r, U(k - q, j, i), g * s[q])
                        if k + 1 + q < nz:
                            put(r, U(k + 1 + q, j, i), -g * s[q])
    n = m.n
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


# ------------------------------------------------------------------ source, receivers
class PointSource3D(PointSource):
    """Ricker point source at the node nearest (sx, sy, sz), sz the depth."""

    def __init__(self, model, sx, sy, sz, f_peak, t0, amp=1.0, p=12):
        i, j, k = (node_index(q, model.dx) for q in (sx, sy, sz))
        if not (0 <= i < model.nx and 0 <= j < model.ny and 0 <= k < model.nz):
            raise ValueError("source outside the grid")
        self.k, self.j, self.i = k, j, i
        self.f_peak, self.t0, self.amp, self.p = f_peak, t0, amp, p
        self.dx = model.dx

    @property
    def node(self):
        return (self.k, self.j, self.i)


def receiver_nodes3d(model, rec):
    """Nearest nodes (k, j, i) of receivers given as (x, y, z) positions."""
    out = []
    for x, y, z in rec:
        i, j, k = (node_index(q, model.dx) for q in (x, y, z))
        if not (0 <= i < model.nx and 0 <= j < model.ny and 0 <= k < model.nz):
            raise ValueError("receiver outside the grid")
        out.append((k, j, i))
    return np.array(out, dtype=np.int64).reshape(-1, 3)


# ------------------------------------------------------------------ leap-frog
def leapfrog3d_init(U):
    u, _v, wx, wy, wz = U
    return (u.copy(), u.copy(), wx.copy(), wx.copy(), wy.copy(), wy.copy(), wz.copy(), wz.copy())


def leapfrog3d_step(m, LF, src, t_n, dt):
    """Sec. 3.1's two-step scheme on the 3D system, damping of w time-averaged and u_t centred
    (the readings of the 2D oracle's default variant)."""
    u, um, wx, wxm, wy, wym, wz, wzm = LF
    bx, by, bz = _betas(m)
    bxh = m.beta_x(True)[None, None, :]
    byh = m.beta_y(True)[None, :, None]
    bzh = m.beta_z(True)[:, None, None]
    b = bx + by + bz
    lap = d_second(m, u, 2) + d_second(m, u, 1) + d_second(m, u, 0)
    div = d_node(m, wx, 2) + d_node(m, wy, 1) + d_node(m, wz, 0)
    rhs = -(bx * by + by * bz + bx * bz) * u + m.c2 * (lap + div)
    if src is not None:
        rhs[src.k, src.j, src.i] += src.f(t_n)
    up = ((2.0 * u - um) / dt ** 2 + b * um / (2.0 * dt) + rhs) / (1.0 / dt ** 2 + b / (2.0 * dt))

    def wnext(wm, bh, g):
        return ((1.0 - bh * dt) * wm + 2.0 * dt * g) / (1.0 + bh * dt)

    wxp = wnext(wxm, bxh, (0.5 * (by + bz) - bxh) * d_half(m, u, 2))
    wyp = wnext(wym, byh, (0.5 * (bx + bz) - byh) * d_half(m, u, 1))
    wzp = wnext(wzm, bzh, (0.5 * (bx + by) - bzh) * d_half(m, u, 0))
    return (up, u, wxp, wx, wyp, wy, wzp, wz)

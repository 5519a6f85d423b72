"""Pins of the oracle's three-dimensional operator and its integrators: two independent routes,
polynomial exactness, symmetry of the Laplacian block, reduction to the 2D operator of Eq. 1 on
a y-invariant field, and convergence to the dense exponential on a tiny grid."""
import math

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import faber, krylov, rk
from oracle import operator as O
from oracle import source as src_mod
from oracle import wave3d as W
from oracle.model import Model, default_beta0, flatten, unflatten
from oracle.simulate import rel_l2
from paper_2401_16322_gb300.workloads import layered, layered3d, smooth_random_state


def _model(nx=11, ny=9, nz=10, pml=3, fs=True, order=8, beta=True, seed=4):
    c = layered3d(nx, ny, nz, seed, vmin=1500, vmax=3000)
    b0 = default_beta0(3000.0, pml, 10.0) if beta else 0.0
    return W.Model3D(nx, ny, nz, 10.0, order, pml, b0, fs, c)


@pytest.mark.parametrize("fs,order", [(True, 8), (False, 8), (False, 4)])
def test_matrix_free_equals_assembled(fs, order):
    m = _model(fs=fs, order=order)
    x = flatten(smooth_random_state(m.field_shapes(), 9))
    a = flatten(W.apply_H3(m, unflatten(m, x)))
    b = W.assemble_H3(m) @ x
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def _poly(deg, t):
    return sum(t ** q / (q + 1) for q in range(deg + 1))


def _dpoly(deg, t):
    return sum(q * t ** (q - 1) / (q + 1) for q in range(1, deg + 1))


def _d2poly(deg, t):
    return sum(q * (q - 1) * t ** (q - 2) / (q + 1) for q in range(2, deg + 1))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_derivatives_exact_for_polynomials_away_from_the_boundary(axis):
    """Interior staggered first derivative exact to degree 7, centred second derivative to
    degree 8, at least R points from any edge.  z (axis 0) is the upward coordinate
    z = -k dx; x and y run with the index."""
    m = _model(nx=20, ny=20, nz=20, fs=False, beta=False)
    dx, R = m.dx, 4
    n = 20
    idx = np.arange(n, dtype=float)
    coord = -idx * dx if axis == 0 else idx * dx
    half = -(idx[:-1] + 0.5) * dx if axis == 0 else (idx[:-1] + 0.5) * dx
    scale = 1.0 / (n * dx)
    shape = [1, 1, 1]
    shape[axis] = n
    f = _poly(7, coord * scale).reshape(shape) * np.ones((n, n, n))
    hshape = [1, 1, 1]
    hshape[axis] = n - 1
    dh = W.d_half(m, f, axis)
    ex = (scale * _dpoly(7, half * scale)).reshape(hshape) * np.ones(dh.shape)
    sl_ = [slice(None)] * 3
    sl_[axis] = slice(R, n - 1 - R)
    assert np.allclose(dh[tuple(sl_)], ex[tuple(sl_)], rtol=1e-10, atol=1e-12)
    # node derivative of a half-point field
    g = _poly(7, half * scale).reshape(hshape) * np.ones(dh.shape)
    dn = W.d_node(m, g, axis)
    exn = (scale * _dpoly(7, coord * scale)).reshape(shape) * np.ones(dn.shape)
    sl_[axis] = slice(R + 1, n - 1 - R)
    assert np.allclose(dn[tuple(sl_)], exn[tuple(sl_)], rtol=1e-10, atol=1e-12)
    # second derivative
    f8 = _poly(8, coord * scale).reshape(shape) * np.ones((n, n, n))
    d2 = W.d_second(m, f8, axis)
    ex2 = (scale ** 2 * _d2poly(8, coord * scale)).reshape(shape) * np.ones(d2.shape)
    sl_[axis] = slice(R, n - R)
    assert np.allclose(d2[tuple(sl_)], ex2[tuple(sl_)], rtol=1e-9, atol=1e-12)


def test_free_surface_rows_exact_for_even_polynomials():
    """Appendix A's top rows in z are exact for polynomials with zero slope at the surface."""
    m = _model(nx=6, ny=5, nz=14, fs=True, beta=False)
    dx = m.dx
    k = np.arange(m.nz, dtype=float)
    z = -k * dx / 100.0
    f = (1.0 + 3 * z ** 2 - 2 * z ** 4 + z ** 6)[:, None, None] * np.ones((m.nz, m.ny, m.nx))
    d2 = W.d_second(m, f, 0)
    ex2 = ((6 - 24 * z ** 2 + 30 * z ** 4) / 100.0 ** 2)[:, None, None]
    assert np.allclose(d2[:4], np.broadcast_to(ex2[:4], d2[:4].shape), rtol=1e-9)
    zh = -(k[:-1] + 0.5) * dx / 100.0
    dh = W.d_half(m, f, 0)
    exh = ((6 * zh - 8 * zh ** 3 + 6 * zh ** 5) / 100.0)[:, None, None]
    assert np.allclose(dh[:3], np.broadcast_to(exh[:3], dh[:3].shape), rtol=1e-9)


def test_laplacian_block_symmetric_without_damping_or_free_surface():
    m = _model(fs=False, beta=False)
    H = W.assemble_H3(m).tocsr()
    N = m.nx * m.ny * m.nz
    c2 = m.c2.ravel()
    L = (H[N:2 * N, :N].toarray()) / c2[:, None]
    assert np.max(np.abs(L - L.T)) <= 1e-12 * np.max(np.abs(L))


def test_reduces_to_the_2d_operator_on_a_y_invariant_field():
    """beta = 0, free surface: for fields constant in y (w_y = 0), the v rows at y rows at
    least R from the y edges equal Eq. 1's 2D operator applied to the x-z slice (z as the 2D
    vertical axis)."""
    nx, ny, nz = 13, 11, 12
    c2d = layered(nx, nz, 7, vmin=1500, vmax=3000)
    c3 = np.repeat(c2d[:, None, :], ny, axis=1)
    m3 = W.Model3D(nx, ny, nz, 10.0, 8, 0, 0.0, True, c3)
    m2 = Model(nx, nz, 10.0, 8, 0, 0.0, True, c2d)
    u2, v2, wx2, wz2 = smooth_random_state(m2.field_shapes(), 21)
    U3 = (np.repeat(u2[:, None, :], ny, 1), np.repeat(v2[:, None, :], ny, 1),
          np.repeat(wx2[:, None, :], ny, 1), np.zeros((nz, ny - 1, nx)),
          np.repeat(wz2[:, None, :], ny, 1))
    h3 = W.apply_H3(m3, U3)
    h2 = O.apply_H(m2, (u2, v2, wx2, wz2))
    for j in range(4, ny - 4):
        assert np.allclose(h3[1][:, j, :], h2[1], rtol=1e-12, atol=1e-12 * np.max(np.abs(h2[1])))
        assert np.array_equal(h3[0][:, j, :], h2[0])


def _dense_aug3(m, s, t, dt):
    H = W.assemble_H3(m).toarray()
    n, p = m.n, s.p
    Ht = np.zeros((n + p, n + p))
    Ht[:n, :n] = H
    N = m.nx * m.ny * m.nz
    Ht[N + (s.k * m.ny + s.j) * m.nx + s.i, n:] = s.W(t, dt)
    for k in range(p - 1):
        Ht[n + k, n + k + 1] = 1.0 / dt
    return Ht


def _tiny3():
    m = _model(nx=8, ny=7, nz=7, pml=2, fs=True)
    s = W.PointSource3D(m, 40.0, 30.0, 20.0, 15.0, 0.05, amp=1.0, p=8)
    U = tuple(smooth_random_state(m.field_shapes(), 5))
    dt, t = 1.2e-3, 0.03
    Ht = _dense_aug3(m, s, t, dt)
    x = np.concatenate([flatten(U), src_mod.e_p(s.p)])
    exact = (sl.expm(dt * Ht) @ x)[:m.n]
    return m, s, U, dt, t, Ht, exact


def test_integrators_converge_to_the_dense_exponential_3d():
    m, s, U, dt, t, Ht, exact = _tiny3()
    params = faber.ellipse_params(m.c_max, m.beta0, m.dx, 8, dims=3, free_surface=True)
    errs = [rel_l2(flatten(faber.faber_step(m, U, s, t, dt, deg, params)), exact) for deg in (10, 40)]
    assert errs[0] > errs[1] and errs[1] < 1e-12
    # MGS in FP64 over 40 vectors: converged to its rounding floor (m = 40 and 60 agree)
    assert rel_l2(flatten(krylov.krylov_step(m, U, s, t, dt, 40)), exact) < 5e-12
    # HORK(m) equals the degree-m Taylor polynomial of exp(dt H~) exactly
    x = np.concatenate([flatten(U), src_mod.e_p(s.p)])
    taylor, term = x.copy(), x.copy()
    for j in range(1, 7):
        term = dt * (Ht @ term) / j
        taylor = taylor + term
    assert rel_l2(flatten(rk.hork_step(m, U, s, t, dt, 6)), taylor[:m.n]) < 1e-13


def test_ellipse_encloses_the_3d_spectrum():
    m = _model(nx=9, ny=8, nz=8, pml=3, fs=True)
    g, c0, c1 = faber.ellipse_params(m.c_max, m.beta0, m.dx, 8, dims=3, free_surface=True)
    ev = np.linalg.eigvals(W.assemble_H3(m).toarray())
    ar, ai = g * (1 + c1), g * (1 - c1)
    assert (((ev.real - g * c0) / ar) ** 2 + (ev.imag / ai) ** 2).max() < 1.0


def test_leapfrog3d_energy_without_damping():
    nx, ny, nz = 10, 9, 9
    m = W.Model3D(nx, ny, nz, 10.0, 8, 0, 0.0, False,
                  layered3d(nx, ny, nz, 3, vmin=1500, vmax=3000))
    u0 = smooth_random_state([(nz, ny, nx)], 4)[0]
    U = (u0,) + tuple(np.zeros(s) for s in m.field_shapes()[1:])
    LF = W.leapfrog3d_init(U)
    dt = 4e-4

    def energy(unp, un):
        Lu = W.d_second(m, un, 0) + W.d_second(m, un, 1) + W.d_second(m, un, 2)
        return 0.5 * np.sum(((unp - un) / dt) ** 2 / m.c2) - 0.5 * np.sum(unp * Lu)

    Es = []
    for n in range(150):
        LF = W.leapfrog3d_step(m, LF, None, n * dt, dt)
        Es.append(energy(LF[0], LF[1]))
    Es = np.array(Es)
    assert np.max(np.abs(Es - Es[0])) <= 1e-10 * np.max(np.abs(Es))


def test_leapfrog3d_second_order():
    """From rest with a Ricker source that starts smoothly (t0 = 2.7 / f), leap-frog converges
    at order 2 to the semi-discrete solution (reference: Faber steps of degree 60, pinned above
    against the dense exponential)."""
    m = _model(nx=8, ny=7, nz=7, pml=2, fs=True)
    s = W.PointSource3D(m, 40.0, 30.0, 20.0, 40.0, 2.7 / 40.0, amp=1.0, p=16)
    T = 0.1
    params = faber.ellipse_params(m.c_max, m.beta0, m.dx, 8, dims=3, free_surface=True)
    U = m.zeros_state()
    nref = 16
    for n in range(nref):
        U = faber.faber_step(m, U, s, n * T / nref, T / nref, 60, params)
    errs = []
    for nst in (160, 320):
        h = T / nst
        LF = W.leapfrog3d_init(m.zeros_state())
        for n in range(nst):
            LF = W.leapfrog3d_step(m, LF, s, n * h, h)
        errs.append(rel_l2(LF[0], U[0]))
    rate = math.log2(errs[0] / errs[1])
    assert abs(rate - 2.0) < 0.15, (errs, rate)

"""Pins of the oracle's operator H (Eq. 1, Secs. 2.1-2.2) against analytic derivatives,
convergence order, energy conservation and an independent sparse assembly."""
import numpy as np
import pytest
import scipy.linalg as sl

from oracle import operator as O
from oracle.model import Model, default_beta0, flatten, unflatten
from paper_2401_16322_gb300.workloads import layered, random_state


def _model(nx, ny, order=8, fs=True, pml=5, c=None, dx=10.0, beta0=None):
    if c is None:
        c = np.full((ny, nx), 2000.0)
    b0 = default_beta0(float(np.max(c)), pml, dx) if beta0 is None else beta0
    return Model(nx, ny, dx, order, pml, b0, fs, c)


@pytest.mark.parametrize("fs,order", [(True, 8), (False, 8), (False, 4)])
def test_matrix_free_equals_assembled(fs, order):
    m = _model(19, 15, order, fs, pml=6, c=layered(19, 15, 11))
    H = O.assemble_H(m)
    for seed in range(3):
        x = random_state([(m.n,)], seed)[0]
        a = flatten(O.apply_H(m, unflatten(m, x)))
        b = H @ x
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))


def _grid(m):
    x = np.arange(m.nx) * m.dx
    y = -np.arange(m.ny) * m.dx           # physical (upward) y, j grows downward
    return x, y


@pytest.mark.parametrize("order", [4, 8])
def test_interior_derivatives_exact_on_polynomials(order):
    """Away from every boundary the stencils differentiate degree <= order polynomials
    exactly (staggered: degree order; centred: degree order+1)."""
    m = _model(30, 28, order, fs=False, pml=0)
    R = order // 2
    x, y = _grid(m)
    X, Y = np.meshgrid(x, y)
    s = 1.0 / (30 * m.dx)
    for deg in range(order + 1):
        u = (X * s) ** deg + 0.5 * (Y * s) ** deg
        ux_exact = deg * (((X[:, :-1] + 0.5 * m.dx) * s) ** max(deg - 1, 0)) * s if deg else 0 * X[:, :-1]
        uyy_exact = 0.5 * deg * (deg - 1) * (Y * s) ** max(deg - 2, 0) * s * s if deg >= 2 else 0 * Y
        uy_exact = 0.5 * deg * (((Y[:-1] - 0.5 * m.dx) * s) ** max(deg - 1, 0)) * s if deg else 0 * Y[:-1]
        sl_i = slice(R + 1, m.nx - R - 2)
        sl_j = slice(R + 1, m.ny - R - 2)
        ux = O.dx_half(m, u)
        assert np.allclose(ux[sl_j, sl_i], ux_exact[sl_j, sl_i], rtol=0, atol=1e-12), deg
        uyy = O.dyy(m, u)
        assert np.allclose(uyy[sl_j, sl_i], uyy_exact[sl_j, sl_i], rtol=0, atol=1e-12), deg
        uy = O.dy_half(m, u)
        assert np.allclose(uy[sl_j, sl_i], uy_exact[sl_j, sl_i], rtol=0, atol=1e-12), deg
        # half -> node derivatives on fields sampled at the half points
        wx = ((X[:, :-1] + 0.5 * m.dx) * s) ** deg
        dwx = O.dx_node(m, wx)
        ex = deg * (X * s) ** max(deg - 1, 0) * s if deg else 0 * X
        assert np.allclose(dwx[sl_j, sl_i], ex[sl_j, sl_i], rtol=0, atol=1e-12), deg
        wy = ((Y[:-1] - 0.5 * m.dx) * s) ** deg
        dwy = O.dy_node(m, wy)
        ey = deg * (Y * s) ** max(deg - 1, 0) * s if deg else 0 * Y
        assert np.allclose(dwy[sl_j, sl_i], ey[sl_j, sl_i], rtol=0, atol=1e-12), deg


def test_free_surface_rows_exact_on_even_polynomials():
    """Rows next to the free surface differentiate u = 1, y^2..y^8 (zero surface slope)
    exactly; d_y w_y rows differentiate w = y..y^8 (w = 0 at the surface) exactly."""
    m = _model(12, 30, 8, fs=True, pml=0)
    x, y = _grid(m)
    X, Y = np.meshgrid(x, y)
    s = 1.0 / (30 * m.dx)
    for deg in [0] + list(range(2, 9)):
        u = (Y * s) ** deg
        uyy = O.dyy(m, u)[:4]
        ex = (deg * (deg - 1) * (Y[:4] * s) ** max(deg - 2, 0) * s * s) if deg >= 2 else 0 * Y[:4]
        assert np.allclose(uyy, ex, rtol=0, atol=1e-12), deg
        uy = O.dy_half(m, u)[:3]
        yh = Y[:3] - 0.5 * m.dx
        ex = deg * (yh * s) ** max(deg - 1, 0) * s if deg else 0 * yh
        assert np.allclose(uy, ex, rtol=0, atol=1e-12), deg
    for deg in range(1, 9):
        wy = ((Y[:-1] - 0.5 * m.dx) * s) ** deg
        dwy = O.dy_node(m, wy)[:4]
        ex = deg * (Y[:4] * s) ** (deg - 1) * s
        assert np.allclose(dwy, ex, rtol=0, atol=1e-12), deg


@pytest.mark.parametrize("order", [4, 8])
def test_convergence_order_on_smooth_wave(order):
    """Error of c^2 Laplacian of sin(kx x) cos(ky y) on the interior falls as dx^order."""
    errs = []
    L = 1000.0
    for n in (40, 80):
        dx = L / n
        m = _model(n + 1, n + 1, order, fs=False, pml=0, dx=dx)
        x = np.arange(m.nx) * dx
        y = -np.arange(m.ny) * dx
        X, Y = np.meshgrid(x, y)
        kx, ky = 2 * np.pi * 3 / L, 2 * np.pi * 2 / L
        u = np.sin(kx * X) * np.cos(ky * Y)
        lap = O.dxx(m, u) + O.dyy(m, u)
        ex = -(kx ** 2 + ky ** 2) * u
        c = slice(n // 4, 3 * n // 4)
        errs.append(np.max(np.abs(lap[c, c] - ex[c, c])) / np.max(np.abs(ex)))
    rate = np.log2(errs[0] / errs[1])
    assert rate > order - 0.3, (errs, rate)


def test_energy_conserved_without_damping():
    """beta = 0, no free surface, w = 0: E = 1/2 v.C^-2 v - 1/2 u.L u is invariant under
    exp(t H) (L symmetric under zero extension)."""
    nx, ny = 13, 11
    c = layered(nx, ny, 4, vmin=1500, vmax=3000)
    m = _model(nx, ny, 8, fs=False, pml=0, c=c, beta0=0.0)
    H = O.assemble_H(m).toarray()
    u, v = random_state([(ny, nx), (ny, nx)], 9)
    U = (u, v, np.zeros((ny, nx - 1)), np.zeros((ny - 1, nx)))

    def energy(U):
        u, v = U[0], U[1]
        Lu = O.dxx(m, u) + O.dyy(m, u)
        return 0.5 * np.sum(v * v / m.c2) - 0.5 * np.sum(u * Lu)

    E0 = energy(U)
    for t in (1e-3, 1e-2, 5e-2):
        Ut = unflatten(m, sl.expm(t * H) @ flatten(U))
        assert abs(energy(Ut) - E0) <= 1e-9 * abs(E0)
    # a sign error in the v-row would break it: flip the Laplacian's sign
    Hbad = H.copy()
    nn = nx * ny
    Hbad[nn:2 * nn, :nn] *= -1.0
    Ut = unflatten(m, sl.expm(5e-2 * Hbad) @ flatten(U))
    assert abs(energy(Ut) - E0) > 1e-3 * abs(E0)


def test_damping_profile_values():
    """beta = beta0 (1 - d/delta)^2: spot values of the boundary-distance reading."""
    m = _model(20, 16, 8, fs=True, pml=4, beta0=100.0)
    bx = m.beta_x_node()
    assert bx[0] == pytest.approx(100.0 * (1 - 1 / 4) ** 2)
    assert bx[3] == pytest.approx(0.0)          # d = 4 = delta -> (1 - 1)^2 = 0
    assert bx[19] == pytest.approx(bx[0])
    assert m.beta_x_half()[0] == pytest.approx(100.0 * (1 - 1.5 / 4) ** 2)
    by = m.beta_y_node()
    assert by[0] == 0.0 and by[15] == pytest.approx(100.0 * (1 - 1 / 4) ** 2)
    m2 = _model(20, 16, 8, fs=False, pml=4, beta0=100.0)
    assert m2.beta_y_node()[0] == pytest.approx(100.0 * (1 - 1 / 4) ** 2)

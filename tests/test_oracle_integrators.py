"""Pins of the oracle's time integrators (Sec. 3) against the dense matrix exponential of
the augmented operator (brute force on tiny grids), library special functions and closed
forms."""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest
import scipy.linalg as sl
import scipy.special as sps

from oracle import faber, krylov, leapfrog, rk
from oracle import operator as O
from oracle import source as src_mod
from oracle.model import Model, default_beta0, flatten, unflatten
from oracle.simulate import rel_l2
from paper_2401_16322_gb300.workloads import layered, smooth_random_state


def _tiny(fs=True, order=8, nx=14, ny=11, pml=4, seed=5):
    c = layered(nx, ny, seed)
    return Model(nx, ny, 10.0, order, pml, default_beta0(c.max(), pml, 10.0), fs, c)


def _dense_aug(m, src, t, dt):
    """Dense H~ (scaled tail) built from the independently assembled sparse H."""
    H = O.assemble_H(m).toarray()
    n, p = m.n, src.p
    Ht = np.zeros((n + p, n + p))
    Ht[:n, :n] = H
    Ht[m.nx * m.ny + src.j * m.nx + src.i, n:] = src.W(t, dt)
    for k in range(p - 1):
        Ht[n + k, n + k + 1] = 1.0 / dt
    return Ht


def _setup(fs=True, order=8, p=8, dt=1.5e-3, t=0.03):
    m = _tiny(fs, order)
    s = src_mod.PointSource(m, 70.0, 20.0 if fs else 50.0, 15.0, 0.05, amp=1.0, p=p)
    U = tuple(smooth_random_state([f.shape for f in m.zeros_state()], 3))
    Ht = _dense_aug(m, s, t, dt)
    x = np.concatenate([flatten(U), src_mod.e_p(p)])
    exact = (sl.expm(dt * Ht) @ x)[:m.n]
    return m, s, U, Ht, x, exact, dt, t


# ----------------------------------------------------------------- source / tail
def test_ricker_derivatives_closed_form():
    sympy = pytest.importorskip("sympy")
    tt = sympy.symbols("t")
    f, t0 = 12.0, 0.2
    a = (sympy.pi * f) ** 2
    r = (1 - 2 * a * (tt - t0) ** 2) * sympy.exp(-a * (tt - t0) ** 2)
    for tv in (0.13, 0.2, 0.26):
        got = src_mod.ricker_derivatives(tv, f, t0, 8)
        for k in range(8):
            ex = float(sympy.diff(r, tt, k).subs(tt, tv))
            assert got[k] == pytest.approx(ex, rel=1e-10, abs=1e-10 * (2 * math.pi * f) ** k)


def test_tail_reproduces_taylor_polynomial_of_source():
    """[0 | W] exp(s J~) e_p = sum_k f^(k)(t_n) s^k/k! (Eq. matrix_ampli's augmentation)."""
    p, dt, tn = 10, 2e-3, 0.1
    J = np.diag(np.ones(p - 1), 1) / dt
    w = src_mod.W_scalars(tn, dt, p, 15.0, 0.12, 1.0, 1.0)
    d = src_mod.ricker_derivatives(tn, 15.0, 0.12, p)
    for s in (0.0, 0.5 * dt, dt):
        y = sl.expm(s * J) @ src_mod.e_p(p)
        taylor = sum(d[k] * s ** k / math.factorial(k) for k in range(p))
        assert float(w @ y) == pytest.approx(taylor, rel=1e-12, abs=1e-14)


def test_node_index_rule():
    assert src_mod.node_index(0.0, 10.0) == 0
    assert src_mod.node_index(14.999, 10.0) == 1
    assert src_mod.node_index(15.0, 10.0) == 2
    assert src_mod.node_index(24.9, 10.0) == 2


# ----------------------------------------------------------------- Faber
@pytest.mark.parametrize("c1", [-0.6, -0.05, 0.3, 1.0])
def test_faber_coefficients_bessel_closed_form(c1):
    dt, gamma, c0, m = 1e-3, 1500.0, -0.3, 40
    a = faber.faber_coefficients(dt, gamma, c0, c1, m)
    x = 2 * dt * gamma * math.sqrt(abs(c1))
    for j in range(m + 1):
        if c1 < 0:
            ex = math.exp(dt * gamma * c0) * sps.jv(j, x) / abs(c1) ** (j / 2)
        else:
            ex = math.exp(dt * gamma * c0) * sps.iv(j, x) / c1 ** (j / 2)
        # round-off of the N-point sum is absolute, on the scale of the largest a_j
        assert a[j] == pytest.approx(ex, rel=1e-11, abs=1e-14 * np.max(np.abs(a)))


def test_faber_coefficients_taylor_case():
    dt, gamma, c0, m = 2e-3, 700.0, -0.2, 20
    a = faber.faber_coefficients(dt, gamma, c0, 0.0, m)
    for j in range(m + 1):
        ex = (dt * gamma) ** j * math.exp(dt * gamma * c0) / math.factorial(j)
        assert a[j] == pytest.approx(ex, rel=1e-11, abs=1e-14 * np.max(np.abs(a)))


@pytest.mark.parametrize("fs", [True, False])
def test_faber_ellipse_encloses_spectrum(fs):
    m = _tiny(fs=fs, order=8, nx=24, ny=18, pml=5, seed=2)
    g, c0, c1 = faber.ellipse_params(m.c_max, m.beta0, m.dx, 8, free_surface=fs)
    ev = np.linalg.eigvals(O.assemble_H(m).toarray())
    ar, ai = g * (1 + c1), g * (1 - c1)
    inside = ((ev.real - g * c0) / ar) ** 2 + (ev.imag / ai) ** 2
    assert inside.max() < 1.0


def test_faber_recurrence_polynomials():
    """F_j(psi(w)) = w^j + c1^j w^-j for the recurrence of Sec. 3.2."""
    g, c0, c1 = 3.0, -0.4, -0.3
    w = np.exp(1j * np.linspace(0, 2 * np.pi, 7)) * 1.3
    z = g * (w + c0 + c1 / w)
    F = [np.ones_like(z), z / g - c0]
    F.append(F[1] * F[1] - 2 * c1)
    for j in range(3, 12):
        F.append(F[1] * F[-1] - c1 * F[-2])
    for j in range(1, 12):
        assert np.allclose(F[j], w ** j + c1 ** j * w ** (-j), rtol=1e-12)


@pytest.mark.parametrize("fs,order", [(True, 8), (False, 4)])
def test_faber_step_converges_to_expm(fs, order):
    m, s, U, Ht, x, exact, dt, t = _setup(fs, order)
    params = faber.ellipse_params(m.c_max, m.beta0, m.dx, order, free_surface=fs)
    errs = [rel_l2(flatten(faber.faber_step(m, U, s, t, dt, deg, params)), exact)
            for deg in (8, 16, 40)]
    assert errs[0] > errs[1]
    assert errs[2] < 1e-12


# ----------------------------------------------------------------- Krylov
def test_expm_against_scipy_and_closed_forms():
    rng = np.random.default_rng(0)
    for scale in (0.1, 1.0, 30.0, 300.0):
        A = rng.standard_normal((12, 12)) * scale / 12
        E = sl.expm(A)
        assert np.max(np.abs(krylov.expm(A) - E)) <= 1e-12 * np.max(np.abs(E))
    th = 2.3
    R = krylov.expm(np.array([[0.0, th], [-th, 0.0]]))
    assert np.allclose(R, [[math.cos(th), math.sin(th)], [-math.sin(th), math.cos(th)]],
                       atol=1e-14)
    N = np.diag(np.ones(4), 1)
    ex = sum(np.linalg.matrix_power(N, k) / math.factorial(k) for k in range(5))
    assert np.allclose(krylov.expm(N), ex, atol=1e-15)
    assert krylov.pade_coefficients(13)[0] == 1.0


def test_arnoldi_relation_and_orthonormality():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((40, 40))
    x = rng.standard_normal(40)
    beta, V, Hm, me = krylov.arnoldi(lambda v: A @ v, x, 10)
    assert me == 10
    assert np.allclose(V.T @ V, np.eye(10), atol=1e-13)
    assert np.allclose(V.T @ A @ V, Hm, atol=1e-12)
    assert np.allclose(np.tril(Hm, -2), 0.0)


def test_incomplete_orthogonalisation_keeps_the_arnoldi_relation():
    """Window q: H is banded (h_kj = 0 for k < j - q + 1, 0-based), the Arnoldi relation
    A V_j = V_{j+1} H_j holds for every column, and a window of m is the full process."""
    rng = np.random.default_rng(2)
    A = rng.standard_normal((40, 40))
    x = rng.standard_normal(40)
    m, q = 10, 2
    beta, V, Hm, me = krylov.arnoldi(lambda v: A @ v, x, m, window=q)
    assert me == m and abs(beta - np.linalg.norm(x)) < 1e-13 * beta
    for j in range(m):
        for k in range(0, max(0, j - q + 1)):
            assert Hm[k, j] == 0.0
    assert np.allclose(A @ V[:, :m - 1], V @ Hm[:, :m - 1], atol=1e-12)
    assert not np.allclose(V.T @ V, np.eye(m), atol=1e-6)      # not orthonormal any more
    full = krylov.arnoldi(lambda v: A @ v, x, m)
    wide = krylov.arnoldi(lambda v: A @ v, x, m, window=m)
    assert np.array_equal(full[1], wide[1]) and np.array_equal(full[2], wide[2])


def test_arnoldi_happy_breakdown():
    A = np.diag(np.arange(1.0, 9.0))
    x = np.zeros(8)
    x[:3] = 1.0                        # lies in a 3-dimensional invariant subspace
    beta, V, Hm, me = krylov.arnoldi(lambda v: A @ v, x, 6)
    assert me == 3
    assert np.allclose(beta * V @ krylov.expm(Hm)[:, 0], sl.expm(A) @ x, rtol=1e-12)


@pytest.mark.parametrize("fs", [True, False])
def test_krylov_step_full_dimension_is_exact(fs):
    m, s, U, Ht, x, exact, dt, t = _setup(fs)
    got = flatten(krylov.krylov_step(m, U, s, t, dt, 60))
    assert rel_l2(got, exact) < 1e-11
    e10 = rel_l2(flatten(krylov.krylov_step(m, U, s, t, dt, 10)), exact)
    assert 1e-14 < e10 < 1e-5


# ----------------------------------------------------------------- RK family
def test_hork_lambdas():
    assert rk.hork_lambdas(4, exact=True) == [Fr(3, 8), Fr(1, 3), Fr(1, 4), Fr(1, 24)]
    for mm in range(1, 15):
        lam = rk.hork_lambdas(mm, exact=True)
        assert sum(lam) == 1 and all(l >= 0 for l in lam)


@pytest.mark.parametrize("mm", [1, 2, 4, 9])
def test_hork_equals_taylor_polynomial(mm):
    m, s, U, Ht, x, exact, dt, t = _setup()
    A = dt * Ht
    T = np.eye(A.shape[0])
    term = np.eye(A.shape[0])
    for j in range(1, mm + 1):
        term = term @ A / j
        T = T + term
    got = flatten(rk.hork_step(m, U, s, t, dt, mm))
    assert rel_l2(got, (T @ x)[:m.n]) < 1e-13


def _stability_poly(coefs, A):
    P = np.zeros_like(A)
    term = np.eye(A.shape[0])
    for c in coefs:
        P = P + c * term
        term = term @ A
    return P


def test_rk32_rk44_stability_polynomials():
    m = _tiny(fs=True)
    H = O.assemble_H(m).toarray()
    U = tuple(smooth_random_state([f.shape for f in m.zeros_state()], 8))
    dt = 1e-3
    x = flatten(U)
    got32 = flatten(rk.rk32_step(m, U, None, 0.0, dt))
    ex32 = _stability_poly([1, 1, 0.5, 0.25], dt * H) @ x
    assert rel_l2(got32, ex32) < 1e-13
    got44 = flatten(rk.rk44_step(m, U, None, 0.0, dt))
    ex44 = _stability_poly([1, 1, 0.5, 1 / 6, 1 / 24], dt * H) @ x
    assert rel_l2(got44, ex44) < 1e-13


_REF_CACHE = {}


def _reference_with_source(m, s, nsteps, dt):
    """Exact semi-discrete solution from zero state with the Ricker source: dense augmented
    exponential with a high-order tail, stepped at dt (the tail is exact to ~1e-16)."""
    key = (m.nx, m.ny, nsteps, dt, s.i, s.j, s.p, s.f_peak, s.t0)
    if key in _REF_CACHE:
        return _REF_CACHE[key]
    H = O.assemble_H(m).toarray()
    x = flatten(m.zeros_state())
    for n in range(nsteps):
        Ht = np.zeros((m.n + s.p, m.n + s.p))
        Ht[:m.n, :m.n] = H
        Ht[m.nx * m.ny + s.j * m.nx + s.i, m.n:] = s.W(n * dt, dt)
        for k in range(s.p - 1):
            Ht[m.n + k, m.n + k + 1] = 1.0 / dt
        xa = np.concatenate([x, src_mod.e_p(s.p)])
        x = (sl.expm(dt * Ht) @ xa)[:m.n]
    _REF_CACHE[key] = x
    return x


@pytest.mark.parametrize("method,order", [("rk32", 2), ("rk44", 4), ("leapfrog", 2)])
def test_low_order_convergence(method, order):
    m = _tiny(fs=True, nx=12, ny=10)
    T = 0.06
    errs = []
    for nsteps in (60, 120):
        dt = T / nsteps
        s = src_mod.PointSource(m, 60.0, 30.0, 25.0, 0.04, p=16)
        ref = _reference_with_source(m, s, nsteps, dt)
        U = m.zeros_state()
        if method == "leapfrog":
            LF = leapfrog.leapfrog_init(U)
            for n in range(nsteps):
                LF = leapfrog.leapfrog_step(m, LF, s, n * dt, dt)
            got = np.concatenate([LF[0].ravel()])
            ref_u = ref[:m.nx * m.ny]
            errs.append(rel_l2(got, ref_u))
        else:
            step = rk.rk32_step if method == "rk32" else rk.rk44_step
            for n in range(nsteps):
                U = step(m, U, s, n * dt, dt)
            errs.append(rel_l2(flatten(U), ref))
    rate = math.log2(errs[0] / errs[1])
    assert abs(rate - order) < 0.35, (errs, rate)


def test_leapfrog_energy_without_damping():
    """beta = 0, no free surface, f = 0: the leap-frog energy
    1/2 |(u^{n+1}-u^n)/dt|^2_{C^-2} - 1/2 (u^{n+1})^T L u^n is conserved to round-off."""
    nx, ny = 15, 13
    c = layered(nx, ny, 3, vmin=1500, vmax=3000)
    m = Model(nx, ny, 10.0, 8, 0, 0.0, False, c)
    u0 = smooth_random_state([(ny, nx)], 4)[0]
    U = (u0, np.zeros((ny, nx)), np.zeros((ny, nx - 1)), np.zeros((ny - 1, nx)))
    LF = leapfrog.leapfrog_init(U)
    dt = 5e-4

    def energy(unp, un):
        Lu = O.dxx(m, un) + O.dyy(m, un)
        return 0.5 * np.sum(((unp - un) / dt) ** 2 / m.c2) - 0.5 * np.sum(unp * Lu)

    Es = []
    for n in range(200):
        LF = leapfrog.leapfrog_step(m, LF, None, n * dt, dt)
        Es.append(energy(LF[0], LF[1]))
    Es = np.array(Es)
    assert np.max(np.abs(Es - Es[0])) <= 1e-10 * np.max(np.abs(Es))


@pytest.mark.parametrize("mm", [1, 3, 8, 16])
def test_horner_recursion_is_the_hork_polynomial(mm):
    """The evaluation order the library offers for HORK: V_{m+1} = x, V_j = x + (dt/j) H~ V_{j+1}
    (j = m .. 1) on the dense augmented operator gives the oracle's HORK step (the paper's
    low-storage stages), i.e. the same degree-m Taylor polynomial."""
    m, s, U, Ht, x, exact, dt, t = _setup()
    V = x.copy()
    for j in range(mm, 0, -1):
        V = x + (dt / j) * (Ht @ V)
    got = flatten(rk.hork_step(m, U, s, t, dt, mm))
    assert rel_l2(got, V[:m.n]) < 1e-13


def test_leapfrog_difference_form_is_the_same_update():
    """The difference form of the averaged leap-frog update: with d = u^n - u^{n-1},
    u^{n+1} = u^n + (d (1 - b dt/2) + dt^2 rhs) / (1 + b dt/2) equals
    ((2u^n - u^{n-1})/dt^2 + b u^{n-1}/(2 dt) + rhs) / (1/dt^2 + b/(2 dt)) for any values."""
    rng = np.random.default_rng(29)
    u, um, rhs = rng.standard_normal((3, 1000))
    b = rng.uniform(0.0, 300.0, 1000)
    dt = rng.uniform(1e-5, 5e-3, 1000)
    plain = ((2 * u - um) / dt ** 2 + b * um / (2 * dt) + rhs) / (1 / dt ** 2 + b / (2 * dt))
    d = u - um
    diff = u + (d * (1 - b * dt / 2) + dt ** 2 * rhs) / (1 + b * dt / 2)
    assert np.allclose(diff, plain, rtol=1e-12, atol=1e-12 * np.abs(plain).max())

"""Pins of the auxiliary-field 3D PML oracle (oracle/wave3d_pml.py): two independent routes,
exact reduction to Eq. 1 with damping on a field that does not vary along an undamped axis,
reduction to the 3D operator without damping, and a stable dense spectrum."""
import numpy as np
import pytest
import scipy.linalg as sl

from oracle import operator as O
from oracle import wave3d as W
from oracle import wave3d_pml as P
from oracle.model import Model, default_beta0, flatten, unflatten
from paper_2401_16322_gb300.workloads import layered, layered3d, smooth_random_state


def _m3(nx=10, ny=9, nz=11, pml=3, fs=True, order=8, beta=True, seed=6):
    c = layered3d(nx, ny, nz, seed, vmin=1500, vmax=3000)
    b0 = default_beta0(3000.0, pml, 10.0) if beta else 0.0
    return W.Model3D(nx, ny, nz, 10.0, order, pml, b0, fs, c)


def _split(m, x):
    out, o = [], 0
    for s in P.field_shapes(m):
        n = int(np.prod(s))
        out.append(x[o:o + n].reshape(s))
        o += n
    return tuple(out)


@pytest.mark.parametrize("fs,order,undamped", [(True, 8, ()), (False, 8, ()), (False, 4, ()),
                                               (True, 8, ("y",))])
def test_matrix_free_equals_assembled(fs, order, undamped):
    m = _m3(fs=fs, order=order)
    x = flatten(smooth_random_state(P.field_shapes(m), 3))
    a = flatten(P.apply_H3p(m, _split(m, x), undamped=undamped))
    b = P.assemble_H3p(m, undamped=undamped) @ x
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_reduces_to_eq1_with_damping_on_a_y_invariant_field():
    """No damping along y and a field constant in y (w_y = 0): on the y rows at least R from
    the y edges, the v, w_x and w_z rows equal Eq. 1's 2D operator on the x-z slice with its
    damping and free-surface rows; w_y stays zero and psi_t = u."""
    nx, ny, nz, pml = 13, 11, 12, 3
    c2d = layered(nx, nz, 7, vmin=1500, vmax=3000)
    b0 = default_beta0(3000.0, pml, 10.0)
    c3 = np.repeat(c2d[:, None, :], ny, axis=1)
    m3 = W.Model3D(nx, ny, nz, 10.0, 8, pml, b0, True, c3)
    m2 = Model(nx, nz, 10.0, 8, pml, b0, True, c2d)
    u2, v2, wx2, wz2 = smooth_random_state(m2.field_shapes(), 21)
    psi = np.repeat(smooth_random_state([(nz, nx)], 22)[0][:, None, :], ny, 1)   # y-invariant
    U3 = (np.repeat(u2[:, None, :], ny, 1), np.repeat(v2[:, None, :], ny, 1),
          np.repeat(wx2[:, None, :], ny, 1), np.zeros((nz, ny - 1, nx)),
          np.repeat(wz2[:, None, :], ny, 1), psi)
    h3 = P.apply_H3p(m3, U3, undamped=("y",))
    h2 = O.apply_H(m2, (u2, v2, wx2, wz2))
    for j in range(4, ny - 4):
        for got, ref in ((h3[1][:, j, :], h2[1]), (h3[2][:, j, :], h2[2]), (h3[4][:, j, :], h2[3])):
            assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.max(np.abs(ref)))
    assert np.array_equal(h3[0], U3[1]) and np.array_equal(h3[5], U3[0])
    assert np.max(np.abs(h3[3][:, 4:ny - 5, :])) == 0.0


def test_mean_reading_does_not_reduce_where_this_one_does():
    """The same y-invariant comparison against oracle.wave3d's mean-of-the-others reading
    fails in the damped layer: the reason this formulation exists."""
    nx, ny, nz, pml = 13, 11, 12, 3
    c2d = layered(nx, nz, 7, vmin=1500, vmax=3000)
    b0 = default_beta0(3000.0, pml, 10.0)
    m3 = W.Model3D(nx, ny, nz, 10.0, 8, pml, b0, True, np.repeat(c2d[:, None, :], ny, axis=1))
    m2 = Model(nx, nz, 10.0, 8, pml, b0, True, c2d)
    u2, v2, wx2, wz2 = smooth_random_state(m2.field_shapes(), 21)
    U3 = (np.repeat(u2[:, None, :], ny, 1), np.repeat(v2[:, None, :], ny, 1),
          np.repeat(wx2[:, None, :], ny, 1), np.zeros((nz, ny - 1, nx)),
          np.repeat(wz2[:, None, :], ny, 1))
    h2 = O.apply_H(m2, (u2, v2, wx2, wz2))
    h3 = W.apply_H3(m3, U3)
    j = ny // 2                                   # interior in y: beta_y = 0 there
    assert not np.allclose(h3[2][:, j, :], h2[2], rtol=1e-6, atol=1e-6 * np.max(np.abs(h2[2])))


def test_without_damping_equals_the_3d_operator():
    m = _m3(beta=False)
    U = tuple(smooth_random_state(P.field_shapes(m), 4))
    hp = P.apply_H3p(m, U)
    h = W.apply_H3(m, U[:5])
    for a, b in zip(hp[:5], h):
        assert np.allclose(a, b, rtol=1e-14, atol=1e-14 * np.max(np.abs(b)))
    assert np.array_equal(hp[5], U[0])


def test_dense_spectrum_is_stable():
    """No growing mode: on a small free-surface cube the largest real part of the dense
    spectrum is at round-off level (2e-13 against beta0 = 1036 s^-1), while the damped modes
    reach Re(lambda) = -529 s^-1."""
    m = _m3(nx=8, ny=7, nz=8, pml=3)
    ev = np.linalg.eigvals(P.assemble_H3p(m).toarray())
    assert ev.real.max() < 1e-9 * m.beta0
    assert ev.real.min() < -0.1 * m.beta0


def _tiny3p():
    """A 8 x 7 x 7 cube on the auxiliary-field PML with a source, a smooth random state (psi
    included) and the dense augmented operator [[H, W], [0, J/dt]] built from assemble_H3p."""
    from oracle import source as src_mod
    nx, ny, nz, pml = 8, 7, 7, 2
    c = layered3d(nx, ny, nz, 5, vmin=1500, vmax=3000)
    m = P.Model3DPML(nx, ny, nz, 10.0, 8, pml, default_beta0(3000.0, pml, 10.0), True, c)
    s = W.PointSource3D(m, 40.0, 30.0, 20.0, 40.0, 0.02, amp=1e3, p=8)
    U = tuple(smooth_random_state(P.field_shapes(m), 8))
    dt, t = 1e-3, 0.012
    n, p = m.n, s.p
    Ht = np.zeros((n + p, n + p))
    Ht[:n, :n] = P.assemble_H3p(m).toarray()
    N = nx * ny * nz
    k, j, i = s.node
    Ht[N + (k * ny + j) * nx + i, n:] = s.W(t, dt)
    for q in range(p - 1):
        Ht[n + q, n + q + 1] = 1.0 / dt
    x = np.concatenate([flatten(U), src_mod.e_p(p)])
    exact = (sl.expm(dt * Ht) @ x)[:n]
    return m, s, U, dt, t, Ht, x, exact


def test_integrators_run_on_the_auxiliary_field_pml():
    """The oracle's integrators reach H through oracle.operator.apply_H, which sends a
    Model3DPML to apply_H3p: Faber and Krylov converge to the dense exponential, and HORK(m)
    is the Taylor polynomial of exp(dt H~)."""
    from oracle import faber, krylov, rk
    from oracle.simulate import rel_l2
    m, s, U, dt, t, Ht, x, exact = _tiny3p()
    assert m.n == sum(int(np.prod(f)) for f in P.field_shapes(m))
    params = faber.ellipse_params(m.c_max, m.beta0, m.dx, 8, dims=3, free_surface=True)
    errs = [rel_l2(flatten(faber.faber_step(m, U, s, t, dt, deg, params)), exact)
            for deg in (10, 40)]
    assert errs[0] > errs[1] and errs[1] < 1e-11
    assert rel_l2(flatten(krylov.krylov_step(m, U, s, t, dt, 40)), exact) < 1e-11
    taylor, term = x.copy(), x.copy()
    for jj in range(1, 7):
        term = dt * (Ht @ term) / jj
        taylor = taylor + term
    assert rel_l2(flatten(rk.hork_step(m, U, s, t, dt, 6)), taylor[:m.n]) < 1e-13


def test_auxiliary_field_pml_absorbs_what_the_mean_reading_reflects():
    """A Gaussian pulse in a homogeneous 24^3 cube with a 6-point PML on every side (Faber 30,
    dt 2 ms, to T = 80 ms, when the pulse has entered the layer): the field left in the
    interior is ~1e-2 of the start with the 3D operator of oracle.wave3d (its w rows take the
    mean of the other two damping profiles, so where one profile is on they see half of it),
    and over 20x less with the auxiliary-field PML."""
    from oracle import faber
    n, pml, dx, c0 = 24, 6, 10.0, 2000.0
    c = np.full((n, n, n), c0)
    b0 = default_beta0(c0, pml, dx)
    z = (np.arange(n) - (n - 1) / 2) * dx
    Z, Y, X = np.meshgrid(z, z, z, indexing="ij")
    u0 = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * 15.0 ** 2))
    inner = (slice(pml, n - pml),) * 3
    params = faber.ellipse_params(c0, b0, dx, 8, dims=3, free_surface=False)
    left = {}
    for name, M in (("mean", W.Model3D), ("aux", P.Model3DPML)):
        m = M(n, n, n, dx, 8, pml, b0, False, c)
        U = (u0.copy(),) + tuple(np.zeros(s) for s in m.field_shapes()[1:])
        for k in range(40):
            U = faber.faber_step(m, U, None, k * 2e-3, 2e-3, 30, params)
        left[name] = np.linalg.norm(U[0][inner]) / np.linalg.norm(u0[inner])
    assert left["mean"] > 5e-3
    assert left["aux"] < 2e-3 and left["aux"] < left["mean"] / 10.0, left


def test_leapfrog_without_damping_equals_the_3d_leapfrog():
    """At beta = 0 the psi terms vanish and the w rows coincide with oracle.wave3d's: the
    auxiliary-field leap-frog advances (u, w) exactly as leapfrog3d_step does."""
    m = _m3(beta=False)
    U = tuple(smooth_random_state(P.field_shapes(m), 41))
    LFp = P.leapfrog3dp_init(U)
    LF = W.leapfrog3d_init(U[:5])
    for n in range(4):
        LFp = P.leapfrog3dp_step(m, LFp, None, n * 4e-4, 4e-4)
        LF = W.leapfrog3d_step(m, LF, None, n * 4e-4, 4e-4)
    for a, b in zip(LFp[:8], LF):
        assert np.allclose(a, b, rtol=1e-13, atol=1e-13 * np.max(np.abs(b)))


def test_leapfrog_reduces_to_the_2d_leapfrog_on_a_y_invariant_field():
    """y undamped, a field constant in y: on the y rows at least R from the y edges the
    auxiliary-field leap-frog advances u, w_x and w_z exactly as the 2D oracle's leap-frog
    (averaged damping) advances u, w_x and w_y on the x-z slice, damping and free surface
    included."""
    from oracle import leapfrog as L2
    nx, ny, nz, pml = 13, 41, 12, 3
    c2d = layered(nx, nz, 7, vmin=1500, vmax=3000)
    b0 = default_beta0(3000.0, pml, 10.0)
    m3 = W.Model3D(nx, ny, nz, 10.0, 8, pml, b0, True, np.repeat(c2d[:, None, :], ny, axis=1))
    m2 = Model(nx, nz, 10.0, 8, pml, b0, True, c2d)
    u2, v2, wx2, wz2 = smooth_random_state(m2.field_shapes(), 23)
    rep = lambda a: np.repeat(a[:, None, :], ny, 1)
    U3 = (rep(u2), rep(v2), rep(wx2), np.zeros((nz, ny - 1, nx)), rep(wz2), np.zeros((nz, ny, nx)))
    LF3 = P.leapfrog3dp_init(U3)
    LF2 = L2.leapfrog_init((u2, v2, wx2, wz2))
    dt = 3e-4
    for n in range(2):
        LF3 = P.leapfrog3dp_step(m3, LF3, None, n * dt, dt, undamped=("y",))
        LF2 = L2.leapfrog_step(m2, LF2, None, n * dt, dt, variant="averaged")
    # the y edges' zero extension makes w_y nonzero near them; its effect spreads at most
    # 2 R cells a step, so the middle row (20 cells in) is still exact after 2 steps
    j = ny // 2
    for got, ref in ((LF3[0][:, j, :], LF2[0]), (LF3[2][:, j, :], LF2[2]), (LF3[6][:, j, :], LF2[4])):
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.max(np.abs(ref)))


def test_leapfrog_converges_at_second_order_to_the_semi_discrete_solution():
    """With damping, free surface and a source: the auxiliary-field leap-frog converges at
    order 2 to Faber steps of degree 60 on the same operator (pinned above against the dense
    exponential), in u and in psi."""
    import math
    from oracle import faber
    from oracle.simulate import rel_l2
    nx, ny, nz, pml = 8, 7, 7, 2
    c = layered3d(nx, ny, nz, 5, vmin=1500, vmax=3000)
    m = P.Model3DPML(nx, ny, nz, 10.0, 8, pml, default_beta0(3000.0, pml, 10.0), True, c)
    s = W.PointSource3D(m, 40.0, 30.0, 20.0, 40.0, 2.7 / 40.0, amp=1.0, p=16)
    T = 0.1
    params = faber.ellipse_params(m.c_max, m.beta0, m.dx, 8, dims=3, free_surface=True)
    U = m.zeros_state()
    nref = 16
    for n in range(nref):
        U = faber.faber_step(m, U, s, n * T / nref, T / nref, 60, params)
    errs, perrs = [], []
    for nst in (160, 320):
        h = T / nst
        LF = P.leapfrog3dp_init(m.zeros_state())
        for n in range(nst):
            LF = P.leapfrog3dp_step(m, LF, s, n * h, h)
        errs.append(rel_l2(LF[0], U[0]))
        perrs.append(rel_l2(LF[8], U[5]))
    for e in (errs, perrs):
        rate = math.log2(e[0] / e[1])
        assert abs(rate - 2.0) < 0.15, (e, rate)

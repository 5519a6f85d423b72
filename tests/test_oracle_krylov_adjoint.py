"""Pins of the oracle's exact discrete Krylov adjoint (oracle/krylov_adjoint.py): the taped
sweep is the Krylov step; one step's adjoint agrees with central differences of the step
(in the state and in m = c^2) to the truncation of the difference quotient; with a
full-dimension basis it is the exact exponential's transpose and Frechet derivative
(scipy, Van Loan's block exponential); the FWI gradient agrees with central differences of
the Krylov misfit, also where the step is far from the exponential."""
import numpy as np
import pytest

from oracle.adjoint import faber_forward, misfit
from oracle.krylov import krylov_step
from oracle.krylov_adjoint import KrylovTape, expm_frechet, krylov_exact_adjoint_step
from oracle.krylov_adjoint import krylov_exact_fwi_gradient
from oracle.model import Model, default_beta0, flatten, unflatten
from oracle.simulate import receiver_nodes
from oracle.source import PointSource
from paper_2401_16322_gb300.workloads import layered, smooth_random_state

NX, NY, DX, PML = 24, 16, 10.0, 4


def _model(c, beta0, nx=NX, ny=NY, pml=PML):
    return Model(nx, ny, DX, 8, pml, beta0, True, c)


def _base():
    c = layered(NX, NY, 23, vmin=1500, vmax=3000)
    return c, default_beta0(3000.0, PML, DX)


def _state(m, seed):
    return flatten(smooth_random_state([f.shape for f in m.zeros_state()], seed))


def _src(m):
    return PointSource(m, 9 * DX, 3 * DX, 30.0, 0.03, amp=1e3, p=8)


@pytest.mark.parametrize("window", [None, 3])
def test_tape_reproduces_krylov_step(window):
    c, beta0 = _base()
    m = _model(c, beta0)
    U = _state(m, 1)
    src = _src(m)
    for mm in (1, 5, 12):
        want = flatten(krylov_step(m, unflatten(m, U), src, 0.02, 1.5e-3, mm, window=window))
        got = KrylovTape(m, U, src, 0.02, 1.5e-3, mm, window=window).out
        assert np.array_equal(got, want), mm


def test_expm_frechet_against_scipy():
    import scipy.linalg as sl
    rng = np.random.default_rng(3)
    X, E = rng.standard_normal((7, 7)), rng.standard_normal((7, 7))
    want = sl.expm_frechet(X, E, compute_expm=False)
    assert np.linalg.norm(expm_frechet(X, E) - want) <= 1e-13 * np.linalg.norm(want)


def _step(m, U, src, t, dt, mm, window=None):
    return KrylovTape(m, U, src, t, dt, mm, window=window).out


@pytest.mark.parametrize("scale", [1.0, 1e-4])
@pytest.mark.parametrize("mm,window", [(1, None), (6, None), (12, None), (12, 2)])
def test_step_adjoint_in_the_state_matches_central_differences(mm, window, scale):
    """<Ubar, dU> = d/deps <ybar, K(U + eps dU)> (the step is nonlinear in U: basis, eta).
    ``scale`` 1e-4: a weak wavefield beside the source (the first steps of a shot), where
    the source column W / eta carries most of the step's dependence on eta."""
    c, beta0 = _base()
    m = _model(c, beta0)
    src = _src(m)
    U, ybar, dU = scale * _state(m, 4), _state(m, 5), scale * _state(m, 6)
    t, dt = 0.02, 1.5e-3
    Ubar, _ = krylov_exact_adjoint_step(m, U, ybar, src, t, dt, mm, window=window)

    def central(eps):
        return float(ybar @ (_step(m, U + eps * dU, src, t, dt, mm, window)
                             - _step(m, U - eps * dU, src, t, dt, mm, window))) / (2 * eps)

    # Richardson: the O(eps^2) term of the central quotient cancels (|dU| ~ |U| here, so
    # the curvature of the one-vector step is not small)
    eps = 1e-3
    fd = (4.0 * central(eps / 2) - central(eps)) / 3.0
    an = float(Ubar @ dU)
    assert abs(fd - an) <= 1e-7 * abs(fd), (fd, an)


@pytest.mark.parametrize("mm,window", [(6, None), (12, None), (12, 2)])
def test_step_adjoint_in_m_matches_central_differences(mm, window):
    c, beta0 = _base()
    m = _model(c, beta0)
    src = _src(m)
    U, ybar = _state(m, 7), _state(m, 8)
    t, dt = 0.02, 1.5e-3
    _, grad = krylov_exact_adjoint_step(m, U, ybar, src, t, dt, mm, window=window)
    c2 = c ** 2
    dm = smooth_random_state([(NY, NX)], 9, sigma_cells=2.0)[0] * 0.01 * c2
    eps = 1e-3
    mp, mn = _model(np.sqrt(c2 + eps * dm), beta0), _model(np.sqrt(c2 - eps * dm), beta0)
    fd = float(ybar @ (_step(mp, U, _src(mp), t, dt, mm, window)
                       - _step(mn, U, _src(mn), t, dt, mm, window))) / (2 * eps)
    an = float(np.sum(grad * dm.ravel()))
    assert abs(fd - an) <= 1e-7 * abs(fd), (fd, an)


def _tiny():
    nx, ny, pml = 9, 7, 3
    c = layered(nx, ny, 17, vmin=1500, vmax=3000)
    return _model(c, default_beta0(3000.0, pml, DX), nx, ny, pml), c


def test_full_dimension_adjoint_is_the_exponential_transpose():
    """With m = n + p the Krylov step is exp(dt H~) itself, for every U, so its exact
    adjoint is exp(dt H)^T ybar (no source: the tail does not reach U)."""
    import scipy.linalg as sl
    from oracle.operator import assemble_H
    m, _ = _tiny()
    U, ybar = _state(m, 11), _state(m, 12)
    dt = 4e-4
    Ubar, _ = krylov_exact_adjoint_step(m, U, ybar, None, 0.0, dt, m.n + 1)
    want = sl.expm(dt * assemble_H(m).toarray()).T @ ybar
    assert np.linalg.norm(Ubar - want) <= 1e-9 * np.linalg.norm(want)


def test_full_dimension_gradient_is_the_frechet_derivative():
    """m = n + p, with a source: <grad, dm> is the Frechet derivative of
    <ybar, [I 0] exp(dt H~(m)) [U; e_p]> along dm (Van Loan's block exponential, scipy)."""
    import scipy.linalg as sl
    from oracle.operator import assemble_H
    m, c = _tiny()
    src = PointSource(m, 4 * DX, 2 * DX, 40.0, 0.02, amp=1e3, p=6)
    U, ybar = _state(m, 13), _state(m, 14)
    dt, t = 3e-4, 0.01
    n, p = m.n, src.p
    _, grad = krylov_exact_adjoint_step(m, U, ybar, src, t, dt, n + p)
    dm = smooth_random_state([(m.ny, m.nx)], 15, sigma_cells=1.5)[0] * 0.1 * c ** 2
    m2 = _model(np.sqrt(c ** 2 + dm), m.beta0, m.nx, m.ny, m.pml)
    E = (assemble_H(m2) - assemble_H(m)).toarray()       # H is affine in c^2
    A = np.zeros((n + p, n + p))
    A[:n, :n] = assemble_H(m).toarray()
    A[m.nx * m.ny + src.j * m.nx + src.i, n:] = src.W(t, dt)
    for k in range(p - 1):
        A[n + k, n + k + 1] = 1.0 / dt
    Ed = np.zeros_like(A)
    Ed[:n, :n] = E
    big = np.zeros((2 * (n + p), 2 * (n + p)))
    big[:n + p, :n + p] = dt * A
    big[:n + p, n + p:] = dt * Ed
    big[n + p:, n + p:] = dt * A
    L = sl.expm(big)[:n + p, n + p:]
    x = np.concatenate([U, np.eye(p)[-1]])
    exact = float(ybar @ (L @ x)[:n])
    got = float(np.sum(grad * dm.ravel()))
    assert abs(got - exact) <= 1e-8 * abs(exact), (got, exact)


def _shots(model):
    rec = np.array([[x * DX, 0.0] for x in range(2, NX - 2, 4)])
    return [(PointSource(model, sx, 2 * DX, 30.0, 0.03, amp=1e3, p=8), receiver_nodes(model, rec))
            for sx in (6 * DX, 17 * DX)]


@pytest.mark.parametrize("mm,window", [(8, None), (8, 2)])
def test_fwi_gradient_matches_central_differences(mm, window):
    """Under-resolved Krylov steps (dt 2 ms at m = 8): the step is far from the exponential,
    and the linearised gradient of oracle.adjoint misses central differences of this misfit by
    about a factor of 10; the exact discrete gradient agrees with them (measured ~1e-11)."""
    c_true, beta0 = _base()
    c0 = np.full((NY, NX), float(c_true.mean()))
    dt, nsteps = 2e-3, 12
    mt = _model(c_true, beta0)
    d_obs = [np.array(s) for s in
             _forward(mt, dt, nsteps, mm, window)]
    J0, grad = krylov_exact_fwi_gradient(_model(c0, beta0), _shots(_model(c0, beta0)), d_obs,
                                         dt, nsteps, mm, window=window)
    assert J0 > 0
    c2 = c0 ** 2
    for seed in (21, 22):
        dm = smooth_random_state([(NY, NX)], seed, sigma_cells=2.0)[0] * 0.01 * c2
        eps = 1e-3
        Jp = misfit(_forward(_model(np.sqrt(c2 + eps * dm), beta0), dt, nsteps, mm, window), d_obs)
        Jm = misfit(_forward(_model(np.sqrt(c2 - eps * dm), beta0), dt, nsteps, mm, window), d_obs)
        fd = (Jp - Jm) / (2 * eps)
        an = float(np.sum(grad * dm))
        assert abs(fd - an) <= 1e-6 * abs(fd), (seed, fd, an)


def _forward(model, dt, nsteps, mm, window):
    """Seismograms of the plain Krylov forward (``krylov_step``) for every shot."""
    if window is None:
        return faber_forward(model, _shots(model), dt, nsteps, mm, None, method="krylov")[1]
    out = []
    for src, rec in _shots(model):
        U, S = unflatten(model, np.zeros(model.n)), []
        for n in range(nsteps):
            U = krylov_step(model, U, src, n * dt, dt, mm, window=window)
            S.append(U[0][rec[:, 0], rec[:, 1]].copy())
        out.append(np.array(S))
    return out


@pytest.mark.parametrize("window", [None, 3])
def test_gram_schmidt_intermediates_are_rebuilt_from_the_basis(window):
    """Before the k-th subtraction of column j the tape's vector equals
    A v_j - sum_{k0 <= i < k} h_ij v_i: the reverse sweep can rebuild it from V, A V and H."""
    c, beta0 = _base()
    m = _model(c, beta0)
    tp = KrylovTape(m, _state(m, 31), _src(m), 0.02, 1.5e-3, 10, window=window)
    V, H = tp.V_full, tp.H_full
    for j in range(tp.m_eff):
        Av = tp.matvec(V[:, j])
        k0 = tp.k0[j]
        for idx, k in enumerate(range(k0, j + 1)):
            rebuilt = Av - sum((H[i, j] * V[:, i] for i in range(k0, k)), np.zeros_like(Av))
            assert np.linalg.norm(rebuilt - tp.ws[j][idx]) <= 1e-12 * np.linalg.norm(Av)

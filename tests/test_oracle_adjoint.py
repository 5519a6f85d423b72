"""Pins of the oracle's discrete adjoint and FWI gradient (m = c^2): the dot-product identity
of one adjoint Faber step and central finite differences of the misfit."""
import numpy as np
import pytest

from oracle.adjoint import (faber_adjoint_step, faber_forward, faber_tape, fwi_gradient,
                            hork_adjoint_step, hork_tape, misfit)
from oracle.faber import ellipse_params
from oracle.model import Model, default_beta0, flatten
from oracle.simulate import receiver_nodes
from oracle.source import PointSource
from paper_2401_16322_gb300.workloads import layered, random_state, smooth_random_state

NX, NY, DX, PML = 30, 20, 10.0, 5


def _model(c, beta0):
    return Model(NX, NY, DX, 8, PML, beta0, True, c)


def _setup():
    c_true = layered(NX, NY, 31, vmin=1500, vmax=3000)
    c0 = np.full((NY, NX), float(c_true.mean()))
    beta0 = default_beta0(3000.0, PML, DX)
    params = ellipse_params(3000.0, beta0, DX, 8, free_surface=True)
    return c_true, c0, beta0, params


def _shots(model):
    rec = np.array([[x * DX, 0.0] for x in range(3, NX - 3, 4)])
    out = []
    for sx in (8 * DX, 21 * DX):
        out.append((PointSource(model, sx, 2 * DX, 30.0, 0.04, amp=1e3, p=10), receiver_nodes(model, rec)))
    return out


def test_adjoint_step_dot_product_identity():
    c_true, c0, beta0, params = _setup()
    m = _model(c0, beta0)
    dU, ybar = (flatten(random_state([f.shape for f in m.zeros_state()], s)) for s in (1, 2))
    dt, deg = 2e-3, 14
    # linear part of the step: no source
    _, AdU = faber_tape(m, dU, None, 0.0, dt, deg, params)
    q0, _ = faber_adjoint_step(m, np.zeros(m.n), ybar, None, 0.0, dt, deg, params)
    lhs, rhs = float(np.dot(AdU, ybar)), float(np.dot(dU, q0))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_hork_adjoint_step_dot_product_identity():
    c_true, c0, beta0, params = _setup()
    m = _model(c0, beta0)
    dU, ybar = (flatten(random_state([f.shape for f in m.zeros_state()], s)) for s in (3, 4))
    dt, deg = 3e-4, 6
    _, AdU = hork_tape(m, dU, None, 0.0, dt, deg)
    q0, _ = hork_adjoint_step(m, np.zeros(m.n), ybar, None, 0.0, dt, deg)
    lhs, rhs = float(np.dot(AdU, ybar)), float(np.dot(dU, q0))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


@pytest.mark.parametrize("method,dt,deg", [("faber", 2e-3, 12), ("hork", 5e-4, 8)])
def test_fwi_gradient_matches_central_differences(method, dt, deg):
    c_true, c0, beta0, params = _setup()
    nsteps = 14
    mt = _model(c_true, beta0)
    _, d_obs = faber_forward(mt, _shots(mt), dt, nsteps, deg, params, method=method)
    m0 = _model(c0, beta0)
    J0, grad = fwi_gradient(m0, _shots(m0), d_obs, dt, nsteps, deg, params, method=method)
    assert J0 > 0
    c2 = c0 ** 2
    for seed in (5, 6, 7):
        dm = smooth_random_state([(NY, NX)], seed, sigma_cells=2.0)[0] * 0.01 * c2
        eps = 1e-3
        mp, mm = _model(np.sqrt(c2 + eps * dm), beta0), _model(np.sqrt(c2 - eps * dm), beta0)
        Jp = misfit(faber_forward(mp, _shots(mp), dt, nsteps, deg, params, method=method)[1], d_obs)
        Jm = misfit(faber_forward(mm, _shots(mm), dt, nsteps, deg, params, method=method)[1], d_obs)
        fd = (Jp - Jm) / (2 * eps)
        an = float(np.sum(grad * dm))
        assert abs(fd - an) <= 1e-6 * abs(fd), (seed, fd, an)


def test_gauss_legendre4_exact_to_degree_7():
    from oracle.adjoint import gauss_legendre4
    t, w = gauss_legendre4()
    for k in range(8):
        assert abs(float(np.sum(w * t ** k)) - 1.0 / (k + 1)) < 1e-15
    assert abs(float(np.sum(w * t ** 8)) - 1.0 / 9.0) > 1e-8     # and not beyond


def _tiny_krylov_model():
    nx, ny, pml = 9, 7, 3
    c = layered(nx, ny, 17, vmin=1500, vmax=3000)
    return Model(nx, ny, DX, 8, pml, default_beta0(3000.0, pml, DX), True, c), c


def test_krylov_adjoint_transport_is_the_exponential_transpose():
    """With a full-dimension basis the adjoint transport is exp(dt H)^T ybar exactly."""
    import scipy.linalg as sl
    from oracle.adjoint import krylov_adjoint_step
    from oracle.operator import assemble_H
    m, _ = _tiny_krylov_model()
    ybar = flatten(smooth_random_state([f.shape for f in m.zeros_state()], 11))
    U = flatten(smooth_random_state([f.shape for f in m.zeros_state()], 12))
    dt = 4e-4
    lam, _ = krylov_adjoint_step(m, U, ybar, None, 0.0, dt, m.n + 1)
    H = assemble_H(m).toarray()
    want = sl.expm(dt * H).T @ ybar
    assert np.linalg.norm(lam - want) <= 1e-10 * np.linalg.norm(want)


def test_krylov_gradient_is_the_frechet_derivative():
    """<grad, dm> equals the exact Frechet derivative of <ybar, [I 0] exp(dt H~(m)) [U; e_p]>
    along dm (Van Loan's block exponential), to the accuracy of 4-point Gauss-Legendre."""
    import scipy.linalg as sl
    from oracle.adjoint import krylov_adjoint_step
    from oracle.operator import assemble_H
    m, c = _tiny_krylov_model()
    src = PointSource(m, 4 * DX, 2 * DX, 40.0, 0.02, amp=1e3, p=6)
    U = flatten(smooth_random_state([f.shape for f in m.zeros_state()], 13))
    ybar = flatten(smooth_random_state([f.shape for f in m.zeros_state()], 14))
    dt, t = 3e-4, 0.01
    n, p = m.n, src.p
    _, grad = krylov_adjoint_step(m, U, ybar, src, t, dt, n + p)
    dm = smooth_random_state([(m.ny, m.nx)], 15, sigma_cells=1.5)[0] * 0.1 * c ** 2
    m2 = Model(m.nx, m.ny, DX, 8, m.pml, m.beta0, True, np.sqrt(c ** 2 + dm))
    E = (assemble_H(m2) - assemble_H(m)).toarray()      # H~ is affine in c^2

    def aug(H):
        A = np.zeros((n + p, n + p))
        A[:n, :n] = H
        nxy = m.nx * m.ny
        A[nxy + src.j * m.nx + src.i, n:] = src.W(t, dt)
        for k in range(p - 1):
            A[n + k, n + k + 1] = 1.0 / dt
        return A

    A = dt * aug(assemble_H(m).toarray())
    Ed = np.zeros_like(A)
    Ed[:n, :n] = dt * E
    big = np.zeros((2 * (n + p), 2 * (n + p)))
    big[:n + p, :n + p] = A
    big[:n + p, n + p:] = Ed
    big[n + p:, n + p:] = A
    L = sl.expm(big)[:n + p, n + p:]
    x = np.concatenate([U, np.eye(p)[-1]])
    exact = float(ybar @ (L @ x)[:n])
    got = float(np.sum(grad * dm.ravel()))
    assert abs(got - exact) <= 1e-6 * abs(exact), (got, exact)


def test_krylov_dense_states_are_the_exponential_at_the_gauss_nodes():
    """With a full-dimension basis the step's dense states are [I 0] exp(tau_q dt H~)[U; e_p]
    at the 4-point Gauss-Legendre nodes (dense expm of the augmented matrix, Eq.
    matrix_ampli); with a short basis the state at tau = 1 is the Krylov step's own result."""
    import scipy.linalg as sl
    from oracle.adjoint import gauss_legendre4, krylov_dense_states
    from oracle.krylov import krylov_step
    from oracle.model import unflatten
    from oracle.operator import assemble_H
    m, c = _tiny_krylov_model()
    src = PointSource(m, 4 * DX, 2 * DX, 40.0, 0.02, amp=1e3, p=6)
    U = flatten(smooth_random_state([f.shape for f in m.zeros_state()], 21))
    dt, t = 3e-4, 0.01
    n, p = m.n, src.p
    A = np.zeros((n + p, n + p))
    A[:n, :n] = assemble_H(m).toarray()
    A[m.nx * m.ny + src.j * m.nx + src.i, n:] = src.W(t, dt)
    for k in range(p - 1):
        A[n + k, n + k + 1] = 1.0 / dt
    x = np.concatenate([U, np.eye(p)[-1]])
    taus = gauss_legendre4()[0]
    got = krylov_dense_states(m, U, src, t, dt, n + p)
    for tau, g in zip(taus, got):
        want = (sl.expm(tau * dt * A) @ x)[:n]
        assert np.linalg.norm(g - want) <= 1e-10 * np.linalg.norm(want), tau
    one = krylov_dense_states(m, U, src, t, dt, 6, taus=[1.0])[0]
    step = flatten(krylov_step(m, unflatten(m, U), src, t, dt, 6))
    assert np.linalg.norm(one - step) <= 1e-13 * np.linalg.norm(step)
    # the dense states are not the endpoint: x(tau) moves with tau
    assert np.linalg.norm(got[0] - got[3]) > 1e-3 * np.linalg.norm(got[3])


def test_krylov_fwi_gradient_matches_central_differences():
    """The linearised Krylov gradient agrees with central differences of the Krylov
    forward to the step's time accuracy (the acceptance level of the FWI gradient)."""
    c_true, c0, beta0, params = _setup()
    dt, deg, nsteps = 1e-3, 14, 10
    mt = _model(c_true, beta0)
    _, d_obs = faber_forward(mt, _shots(mt), dt, nsteps, deg, params, method="krylov")
    m0 = _model(c0, beta0)
    J0, grad = fwi_gradient(m0, _shots(m0), d_obs, dt, nsteps, deg, params, method="krylov")
    c2 = c0 ** 2
    for seed in (5, 6):
        dm = smooth_random_state([(NY, NX)], seed, sigma_cells=2.0)[0] * 0.01 * c2
        eps = 1e-3
        mp, mm = _model(np.sqrt(c2 + eps * dm), beta0), _model(np.sqrt(c2 - eps * dm), beta0)
        Jp = misfit(faber_forward(mp, _shots(mp), dt, nsteps, deg, params, method="krylov")[1], d_obs)
        Jm = misfit(faber_forward(mm, _shots(mm), dt, nsteps, deg, params, method="krylov")[1], d_obs)
        fd = (Jp - Jm) / (2 * eps)
        an = float(np.sum(grad * dm))
        assert abs(fd - an) <= 1e-3 * abs(fd), (seed, fd, an)


def test_checkpoint_stride_is_the_smallest_stride_within_budget():
    """Brute force: storing the states at steps 0, s, 2s, ... (those below nsteps) keeps at
    most ``budget`` of them, and no smaller stride does (stride 1 when everything fits)."""
    from oracle.adjoint import checkpoint_stride

    def stored(n, s):
        return len(range(0, n, s))

    for n in range(0, 80):
        for b in range(1, 30):
            s = checkpoint_stride(n, b)
            assert s >= 1 and stored(n, s) <= b, (n, b, s)
            assert s == 1 or stored(n, s - 1) > b, (n, b, s)

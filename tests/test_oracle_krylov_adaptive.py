"""Pins of the oracle's adaptive Krylov step (oracle/krylov_adaptive.py): the phi-function
block against closed forms, the error estimate against the true error, the whole step
against the dense exponential (scipy) within the tolerance, the reduction to the fixed-m
step, exactness on an invariant subspace, and a dimension no larger than the smallest
fixed m that meets the tolerance."""
import numpy as np
import pytest
import scipy.linalg as sl

from oracle.krylov import arnoldi, krylov_step
from oracle.krylov_adaptive import adaptive_exp, error_estimate, krylov_adaptive_step, phi_block
from oracle.model import Model, default_beta0, flatten
from oracle.operator import assemble_H
from oracle.source import PointSource
from paper_2401_16322_gb300.workloads import layered, smooth_random_state

DX = 10.0


def _setup():
    nx, ny, pml = 12, 9, 3
    c = layered(nx, ny, 17, vmin=1500, vmax=3000)
    m = Model(nx, ny, DX, 8, pml, default_beta0(3000.0, pml, DX), True, c)
    src = PointSource(m, 5 * DX, 2 * DX, 40.0, 0.02, amp=1e3, p=6)
    U = smooth_random_state([f.shape for f in m.zeros_state()], 3)
    return m, src, U


def _dense_step(m, src, U, t, dt):
    """[I 0] exp(dt H~) [U; e_p] from the assembled H and the augmented block (scipy)."""
    n, p = m.n, src.p
    A = np.zeros((n + p, n + p))
    A[:n, :n] = assemble_H(m).toarray()
    A[m.nx * m.ny + src.j * m.nx + src.i, n:] = src.W(t, dt)
    for k in range(p - 1):
        A[n + k, n + k + 1] = 1.0 / dt
    return (sl.expm(dt * A) @ np.concatenate([flatten(U), np.eye(p)[-1]]))[:n]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_phi_block_closed_forms():
    """tau phi_1(tau H) e_1 = H^-1 (e^{tau H} - I) e_1 and
    tau^2 phi_2(tau H) e_1 = H^-2 (e^{tau H} - I - tau H) e_1 for invertible H."""
    rng = np.random.default_rng(1)
    H = rng.standard_normal((6, 6)) + 3.0 * np.eye(6)
    tau = 0.7
    E = sl.expm(tau * H)
    I = np.eye(6)
    e, p1, p2 = phi_block(H, tau)
    Hi = np.linalg.inv(H)
    assert _rel(e, E[:, 0]) < 1e-13
    assert _rel(p1, (Hi @ (E - I))[:, 0]) < 1e-12
    assert _rel(p2, (Hi @ Hi @ (E - I - tau * H))[:, 0]) < 1e-11


def _estimate_and_truth(matvec, A_dense, x, j, tau):
    beta, V, H, _ = arnoldi(matvec, x, j + 1)
    e, p1, p2 = phi_block(H[:j, :j], tau)
    est = error_estimate(beta, H[j, j - 1], p1, p2, float(np.linalg.norm(matvec(V[:, j]))))
    true = float(np.linalg.norm(sl.expm(tau * A_dense) @ x - beta * V[:, :j] @ e))
    return est, true


def test_estimate_tracks_the_true_error():
    """Above round-off the two-term estimate lies between the true error and 2.5 times it,
    on a random matrix and on the augmented PML operator with its source column."""
    rng = np.random.default_rng(0)
    n = 60
    A = rng.standard_normal((n, n)) / np.sqrt(n) - 0.3 * np.eye(n)
    x = rng.standard_normal(n)
    for tau in (0.5, 1.0, 2.0):
        for j in (4, 8, 12):
            est, true = _estimate_and_truth(lambda v: A @ v, A, x, j, tau)
            assert true < est <= 2.5 * true, (tau, j, est, true)
    m, src, U = _setup()
    dt, t = 8e-3, 0.01
    n, p = m.n, src.p
    eta = float(np.linalg.norm(flatten(U)))
    Aw = np.zeros((n + p, n + p))
    Aw[:n, :n] = assemble_H(m).toarray()
    Aw[m.nx * m.ny + src.j * m.nx + src.i, n:] = src.W(t, dt) / eta
    for k in range(p - 1):
        Aw[n + k, n + k + 1] = 1.0 / dt
    Aw *= dt
    xw = np.concatenate([flatten(U), eta * np.eye(p)[-1]])
    for tau in (0.25, 0.5, 1.0):
        for j in (6, 10):
            est, true = _estimate_and_truth(lambda v: Aw @ v, Aw, xw, j, tau)
            assert true < est <= 2.5 * true, (tau, j, est, true)


@pytest.mark.parametrize("dt", [2e-3, 8e-3])
@pytest.mark.parametrize("tol", [1e-3, 1e-6, 1e-9])
@pytest.mark.parametrize("m_max,window", [(10, None), (30, None), (30, 4)])
def test_step_matches_dense_exponential(dt, tol, m_max, window):
    m, src, U = _setup()
    t = 0.01
    exact = _dense_step(m, src, U, t, dt)
    got, info = krylov_adaptive_step(m, U, src, t, dt, tol, m_max=m_max, window=window)
    assert _rel(flatten(got), exact) <= 3.0 * tol, info
    assert abs(sum(info["taus"]) - 1.0) < 1e-12
    assert max(info["dims"]) <= m_max


def test_forced_substeps_compose():
    """Starting from tau = 0.05 of the step, the substeps still compose to exp(dt H~)."""
    m, src, U = _setup()
    t, dt, tol = 0.01, 4e-3, 1e-8
    got, info = krylov_adaptive_step(m, U, src, t, dt, tol, m_max=20, tau0=0.05)
    assert info["substeps"] >= 3 and info["taus"][0] == 0.05
    assert _rel(flatten(got), _dense_step(m, src, U, t, dt)) <= 3.0 * tol


def test_zero_state_step_is_the_source_response():
    """From U = 0 the start vector is the tail e_p (norm 1), and the tolerance is relative
    to it: the absolute error of the source response stays within 3 tol."""
    m, src, _ = _setup()
    U0 = m.zeros_state()
    t, dt, tol = 0.01, 4e-3, 1e-8
    got, _ = krylov_adaptive_step(m, U0, src, t, dt, tol, m_max=30)
    assert np.linalg.norm(flatten(got) - _dense_step(m, src, U0, t, dt)) <= 3.0 * tol


@pytest.mark.parametrize("mm,window", [(1, None), (5, None), (12, None), (12, 3)])
def test_reduces_to_the_fixed_dimension_step(mm, window):
    """m_min = m_max = m and no error control: one substep of dimension m, the fixed-m step
    (with the same incomplete-orthogonalisation window)."""
    m, src, U = _setup()
    got, info = krylov_adaptive_step(m, U, src, 0.01, 4e-3, np.inf, m_min=mm, m_max=mm,
                                     window=window)
    assert info["dims"] == [mm] and info["substeps"] == 1
    want = krylov_step(m, U, src, 0.01, 4e-3, mm, window=window)
    assert _rel(flatten(got), flatten(want)) < 1e-13


def test_invariant_subspace_is_exact_in_one_substep():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((8, 8))
    A[3:, :3] = 0.0                      # span(e_1, e_2, e_3) is invariant
    x = np.zeros(8)
    x[:3] = rng.standard_normal(3)
    got, info = adaptive_exp(lambda v: A @ v, x, 1e-12, m_max=6)
    assert info["dims"] == [3] and info["substeps"] == 1
    assert _rel(got, sl.expm(A) @ x) < 1e-12


@pytest.mark.parametrize("tol", [1e-4, 1e-8])
def test_dimension_is_no_larger_than_needed(tol):
    """One substep (m_max large): the chosen dimension is at most one above the smallest
    fixed m whose step already meets the tolerance (relative to the start vector
    [U; |U| e_p], as the control measures it), and not below it by more than one."""
    m, src, U = _setup()
    t, dt = 0.01, 4e-3
    exact = _dense_step(m, src, U, t, dt)
    got, info = krylov_adaptive_step(m, U, src, t, dt, tol, m_max=40)
    assert info["substeps"] == 1
    j = info["dims"][0]
    ref = np.sqrt(2.0) * np.linalg.norm(flatten(U))
    need = next(k for k in range(1, 41)
                if np.linalg.norm(flatten(krylov_step(m, U, src, t, dt, k)) - exact) <= tol * ref)
    assert need - 1 <= j <= need + 1, (j, need)

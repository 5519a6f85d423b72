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

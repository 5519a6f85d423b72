"""Pins of the leap-frog adjoint oracle (oracle/leapfrog_adjoint.py): the assembled step equals
the matrix-free leap-frog step, its forward gives the same seismograms as the oracle's time
loop, and its FWI gradient equals central differences of the misfit computed with that loop."""
import numpy as np
import pytest

from oracle import leapfrog as LF
from oracle import leapfrog_adjoint as LA
from oracle.model import Model, default_beta0
from oracle.simulate import receiver_nodes, run
from oracle.source import PointSource
from paper_2401_16322_gb300.workloads import layered, smooth_random_state

NX, NY, DX, PML = 19, 14, 10.0, 4


def _model(c, fs=True):
    return Model(NX, NY, DX, 8, PML, default_beta0(3000.0, PML, DX), fs, c)


def _shots(m):
    rec = np.array([[x * DX, 0.0] for x in range(2, NX - 2, 3)])
    return [(PointSource(m, sx, 2 * DX, 40.0, 0.03, amp=1e3, p=4), receiver_nodes(m, rec))
            for sx in (6 * DX, 12 * DX)]


@pytest.mark.parametrize("fs", [True, False])
def test_assembled_step_equals_leapfrog_step(fs):
    m = _model(layered(NX, NY, 3, vmin=1500, vmax=3000), fs)
    dt = 6e-4
    A, _ = LA.step_matrix(m, dt)
    sh = [(NY, NX), (NY, NX), (NY, NX - 1), (NY, NX - 1), (NY - 1, NX), (NY - 1, NX)]
    lf = tuple(smooth_random_state(sh, 5))
    got = A @ LA.pack(m, lf)
    ref = LA.pack(m, LF.leapfrog_step(m, lf, None, 0.0, dt))
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_forward_equals_the_oracle_time_loop():
    m = _model(layered(NX, NY, 3, vmin=1500, vmax=3000))
    dt, nsteps = 6e-4, 40
    _, seis = LA.forward(m, _shots(m), dt, nsteps)
    for (src, rn), S in zip(_shots(m), seis):
        _, ref = run(m, "leapfrog", dt, nsteps, src=src, rec_nodes=rn)
        assert np.max(np.abs(S - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_leapfrog_fwi_gradient_matches_central_differences():
    c_true = layered(NX, NY, 31, vmin=1500, vmax=3000)
    c0 = np.full((NY, NX), float(c_true.mean()))
    dt, nsteps = 6e-4, 60
    mt = _model(c_true)
    d_obs = [run(mt, "leapfrog", dt, nsteps, src=s, rec_nodes=rn)[1] for s, rn in _shots(mt)]
    m0 = _model(c0)
    J0, grad = LA.fwi_gradient(m0, _shots(m0), d_obs, dt, nsteps)
    assert J0 > 0

    def J(c2):
        m = _model(np.sqrt(c2))
        return 0.5 * sum(float(np.sum((run(m, "leapfrog", dt, nsteps, src=s, rec_nodes=rn)[1] - d) ** 2))
                         for (s, rn), d in zip(_shots(m), d_obs))

    c2 = c0 ** 2
    for seed in (5, 6):
        dm = smooth_random_state([(NY, NX)], seed, sigma_cells=2.0)[0] * 0.01 * c2
        eps = 1e-3
        fd = (J(c2 + eps * dm) - J(c2 - eps * dm)) / (2 * eps)
        an = float(np.sum(grad * dm))
        assert abs(fd - an) <= 1e-6 * abs(fd), (seed, fd, an)

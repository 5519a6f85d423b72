"""The adaptive Krylov step on the GPU (ewv_step_krylov_adaptive) against the oracle's
(oracle/krylov_adaptive.py, the KIOPS-style reading of Secs. 3.2 and 6): same substeps and
dimensions, and the same state to rounding, in FP64 over tolerances 1e-3 .. 1e-9, with and
without forced substeps, an orthogonalisation window and a batch of two models whose shots
take different substeps."""
import numpy as np
import pytest

from _helpers import flatten, oracle_model, rel_l2
from oracle.krylov_adaptive import krylov_adaptive_step
from oracle.source import PointSource
from paper_2401_16322_gb300.workloads import layered, smooth_random_state

pytestmark = pytest.mark.gpu

NX, NY, P = 40, 30, 8


def _case(seed=4, nx=NX, ny=NY):
    from paper_2401_16322_gb300 import Model
    om = oracle_model(nx, ny, layered(nx, ny, seed), pml=6, fs=True)
    g = Model(om.nx, om.ny, om.dx, 8, om.pml, om.beta0, True, precision="f64", p=P)
    g.set_velocity(om.c)
    sx, sy = (nx // 2) * om.dx + 3.0, 2 * om.dx
    g.set_source_receivers(0, sx, sy, 30.0, 0.04, 1e3, None)
    src = PointSource(om, sx, sy, 30.0, 0.04, amp=1e3, p=P)
    U = smooth_random_state([f.shape for f in om.zeros_state()], seed + 10)
    U = (U[0],) + tuple(0 * f for f in U[1:])          # displacement at rest
    return om, g, src, U


@pytest.mark.parametrize("tol,dt,m_max,window", [(1e-3, 2e-3, 30, 0), (1e-6, 2e-3, 30, 0),
                                                 (1e-9, 2e-3, 30, 0), (1e-6, 8e-3, 30, 0),
                                                 (1e-6, 8e-3, 8, 0), (1e-6, 2e-3, 30, 3)])
def test_adaptive_step_matches_oracle(tol, dt, m_max, window):
    om, g, src, U = _case()
    g.set_krylov_window(window)
    g.set_state(0, flatten(U))
    st = g.step_krylov_adaptive(0.03, dt, tol, 1, m_max, 1)
    g.sync()
    ref, info = krylov_adaptive_step(om, U, src, 0.03, dt, tol, 1, m_max, window=window or None)
    assert st["substeps"] == info["substeps"], (st, info)
    assert st["max_dim"] == max(info["dims"]), (st, info)
    assert rel_l2(g.get_state(0), flatten(ref)) < 1e-10
    if m_max == 8:
        assert info["substeps"] > 1                   # the case forces substeps
    g.close()


def test_adaptive_batch_of_two_models_and_two_steps():
    """Two uneven models in one batch; each shot takes its own substeps, over two steps."""
    from paper_2401_16322_gb300 import Batch
    cases = [_case(4), _case(7, nx=52, ny=27)]
    B = Batch([c[1] for c in cases])
    for om, g, src, U in cases:
        g.set_state(0, flatten(U))
    B.step_krylov_adaptive(0.03, 6e-3, 1e-7, 1, 10, 2)
    B.sync()
    for om, g, src, U in cases:
        ref = U
        for n in range(2):
            ref, _ = krylov_adaptive_step(om, ref, src, 0.03 + n * 6e-3, 6e-3, 1e-7, 1, 10)
        assert rel_l2(g.get_state(0), flatten(ref)) < 1e-10
    B.close()

"""Failure detection on the GPU without a GPU fault.

* A non-finite value planted in the state from the host (ewv_set_state) is caught by the
  end-of-call scan: a Faber or HORK step returns at once (it only enqueues), and the next
  call on the handle, or ewv_sync, reports EWV_ERR_NONFINITE; a Krylov step with an info
  pointer reports it itself (its Arnoldi process sees the value).  After the report the
  handle works again.
* A TMA pipeline wait that gives up: the testing knob ewv_debug_set_wait_limit(0) makes every
  wait of the 2D FP32 pass that is not already satisfied give up at once.  The kernel then
  drains its copies in flight (up to 1 s), sets the timeout bit and returns; the call
  reports EWV_ERR_TIMEOUT, and with the default limit restored the next step is correct.
Nothing here hangs or faults the GPU: every wait in the kernels is bounded."""
import numpy as np
import pytest

from _helpers import TOL, flatten, gpu_model, oracle_ellipse, oracle_model, rel_l2
from oracle.simulate import run
from oracle.source import PointSource
from paper_2401_16322_gb300.workloads import layered, smooth_random_state

pytestmark = pytest.mark.gpu

NX, NY = 83, 37


def _setup(prec):
    om = oracle_model(NX, NY, layered(NX, NY, 4), pml=10, fs=True)
    g = gpu_model(om, prec, p=10)
    g.set_faber_ellipse(*oracle_ellipse(om))
    U0 = tuple(smooth_random_state([f.shape for f in om.zeros_state()], 9))
    return om, g, U0


def _plant_nan(om, U0, value=np.nan):
    x = flatten(U0).copy()
    x[om.nx * 20 + 40] = value               # u at (i = 40, j = 20)
    return x


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("method,m", [("faber", 12), ("hork", 8)])
def test_nonfinite_state_is_reported_by_the_next_call(prec, method, m):
    from paper_2401_16322_gb300.ewave import EwaveError
    om, g, U0 = _setup(prec)
    g.ensure_workspace(method, m)
    g.set_state(0, _plant_nan(om, U0))
    g.step(method, 0.03, 1.2e-3, m, 2)          # enqueues only: no error yet
    with pytest.raises(EwaveError, match="NONFINITE"):
        g.sync()
    g.sync()                                     # the report cleared the word
    # an infinity is caught the same way, this time by the next step call
    g.set_state(0, _plant_nan(om, U0, np.inf))
    g.step(method, 0.03, 1.2e-3, m, 1)
    g.stream.synchronize()
    with pytest.raises(EwaveError, match="NONFINITE"):
        g.step(method, 0.03, 1.2e-3, m, 1)
    # a finite state steps normally afterwards and matches the oracle
    g.set_state(0, flatten(U0))
    g.step(method, 0.03, 1.2e-3, m, 2)
    g.sync()
    U, _ = run(om, method, 1.2e-3, 2, m=m, U0=U0, t0=0.03, faber_params=oracle_ellipse(om))
    assert rel_l2(g.get_state(0), flatten(U)) < TOL[prec] * 2
    g.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_nonfinite_state_in_krylov(prec):
    from paper_2401_16322_gb300 import Batch
    from paper_2401_16322_gb300.ewave import EwaveError
    om, g, U0 = _setup(prec)
    g.ensure_workspace("krylov", 8)
    g.set_state(0, _plant_nan(om, U0))
    with pytest.raises(EwaveError, match="NONFINITE"):
        g.step("krylov", 0.03, 1.2e-3, 8, 1)     # with info: reported by the call itself
    g.sync()
    g.set_state(0, _plant_nan(om, U0))
    B = Batch([g])
    with pytest.raises(EwaveError, match="NONFINITE"):
        B.step("krylov", 0.03, 1.2e-3, 8, 1)
    B.sync()
    B.close()
    g.close()


def test_host_rejects_non_finite_velocity():
    from paper_2401_16322_gb300.ewave import EwaveError
    om, g, _ = _setup("f32")
    c = om.c.copy()
    c[3, 4] = np.nan
    with pytest.raises(EwaveError, match="INVALID_ARG"):
        g.set_velocity(c)
    g.close()


def test_pipeline_wait_timeout_is_reported_and_the_next_call_recovers():
    import torch
    from paper_2401_16322_gb300.ewave import EwaveError, debug_set_wait_limit
    om, g, U0 = _setup("f32")
    src = PointSource(om, 41 * om.dx, 2 * om.dx, 25.0, 0.05, amp=1e3, p=10)
    g.set_source_receivers(0, 41 * om.dx, 2 * om.dx, 25.0, 0.05, 1e3, None)
    g.ensure_workspace("faber", 12)
    g.set_state(0, flatten(U0))
    g.step("faber", 0.03, 1.2e-3, 12, 2)           # tiling tuned, step graph captured
    g.sync()
    try:
        debug_set_wait_limit(0)
        g.set_state(0, flatten(U0))
        g.step("faber", 0.03, 1.2e-3, 12, 2)
        with pytest.raises(EwaveError, match="TIMEOUT"):
            g.sync()
    finally:
        debug_set_wait_limit(1_000_000_000)
    torch.cuda.synchronize()
    g.set_state(0, flatten(U0))
    g.step("faber", 0.03, 1.2e-3, 12, 2)
    g.sync()
    U, _ = run(om, "faber", 1.2e-3, 2, src=src, m=12, U0=U0, t0=0.03,
               faber_params=oracle_ellipse(om))
    assert rel_l2(g.get_state(0), flatten(U)) < TOL["f32"] * 2
    g.close()

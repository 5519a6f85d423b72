"""CUDA-graph replay of the step loop gives bit-identical states and seismograms to direct
launches, for every integrator (leap-frog alternates two captured sequences).  Both runs use
the same FP32 pass variant: the variants' unrolled loops agree to rounding, not bitwise."""
import numpy as np
import pytest

from _helpers import flatten, gpu_model, oracle_ellipse, oracle_model
from paper_2401_16322_gb300.workloads import layered, smooth_random_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("method,m", [("faber", 16), ("hork", 5), ("rk32", 0), ("rk44", 0),
                                      ("krylov", 8), ("leapfrog", 0)])
def test_graph_replay_is_bitwise_identical(prec, method, m):
    nx, ny = 83, 37
    om = oracle_model(nx, ny, layered(nx, ny, 17), pml=10, fs=True)
    rec = np.array([[x * om.dx, 0.0] for x in range(2, nx - 2, 9)])
    U0 = tuple(smooth_random_state([f.shape for f in om.zeros_state()], 12))
    if method == "krylov":
        U0 = (U0[0], 0 * U0[1], 0 * U0[2], 0 * U0[3])
    out = []
    for graphs in (False, True):
        g = gpu_model(om, prec, p=8, max_receivers=len(rec))
        g.set_source_receivers(0, 41 * om.dx, 2 * om.dx, 25.0, 0.05, 1e3, rec)
        g.set_faber_ellipse(*oracle_ellipse(om))
        g.enable_graphs(graphs)
        if prec == "f32":
            g.set_kernel_variant(0)
        g.bind_seismogram(7)
        g.set_state(0, flatten(U0))
        dt = 4e-4 if method == "leapfrog" else 1.1e-3
        g.step(method, 0.03, dt, m, 7)
        out.append((g.get_state(0), g.seismogram(0, len(rec), 7)))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_kernel_timing_inside_replayed_graphs(prec):
    """With graphs and pass timing both on, every pass of every step is timed (external
    event nodes in the captured step) and the states equal those of an untimed run."""
    nx, ny = 83, 37
    om = oracle_model(nx, ny, layered(nx, ny, 17), pml=10, fs=True)
    U0 = tuple(smooth_random_state([f.shape for f in om.zeros_state()], 13))
    out = []
    for timed in (False, True):
        g = gpu_model(om, prec, p=8, max_receivers=1)
        g.set_source_receivers(0, 41 * om.dx, 2 * om.dx, 25.0, 0.05, 1e3, np.array([[0.0, 0.0]]))
        g.set_faber_ellipse(*oracle_ellipse(om))
        if prec == "f32":
            g.set_kernel_variant(0)
        g.enable_graphs(True)
        g.set_state(0, flatten(U0))
        g.enable_kernel_timing(timed)
        g.step("faber", 0.03, 1.1e-3, 12, 6)
        if timed:
            ms, n = g.kernel_timing()
            assert n == 6 * 12 and ms > 0.0
        out.append(g.get_state(0))
    assert np.array_equal(out[0], out[1])


def test_graph_from_an_earlier_call_is_replayed_bit_exactly():
    """A step graph captured in one call is replayed from the first step of the next call
    (one-step calls, as the FWI forward makes): the result equals direct launches."""
    nx, ny = 83, 37
    om = oracle_model(nx, ny, layered(nx, ny, 17), pml=10, fs=True)
    rec = np.array([[x * om.dx, 0.0] for x in range(2, nx - 2, 9)])
    U0 = tuple(smooth_random_state([f.shape for f in om.zeros_state()], 12))
    out = []
    for graphs in (True, False):
        g = gpu_model(om, "f32", p=8, max_receivers=len(rec))
        g.set_source_receivers(0, 41 * om.dx, 2 * om.dx, 25.0, 0.05, 1e3, rec)
        g.enable_graphs(graphs)
        g.set_kernel_variant(0)
        g.bind_seismogram(1)
        g.set_state(0, flatten(U0))
        for n in range(4):
            g.step("hork", 0.03 + n * 1.1e-3, 1.1e-3, 6, 1)
        out.append(g.get_state(0))
    assert np.array_equal(out[0], out[1])

"""The Gram-Schmidt column kernel (one cooperative launch per Arnoldi column, q_{j+1} in
shared memory, a bounded grid barrier per step) against the flat passes it replaces: in FP32
(where the flat form also takes the first dot in a flat pass) the two give the same Krylov
states and seismograms bit for bit, for one model's shots, for uneven models in a batch,
with an orthogonalisation window, with two chunks per block, and in the exponential Krylov
adjoint; in FP64 the flat form fuses the first dot into the stencil pass (another summation
order), so the two agree to rounding; both match the oracle.  A barrier wait that gives up
is reported as EWV_ERR_TIMEOUT and the next call is correct."""
import numpy as np
import pytest

from _helpers import TOL, flatten, gpu_model, oracle_model, rel_l2
from oracle.krylov import krylov_step
from oracle.model import unflatten
from oracle.source import PointSource
from paper_2401_16322_gb300.workloads import layered, smooth_random_state

pytestmark = pytest.mark.gpu

DT, T0 = 1.5e-3, 0.03
VARIANT = 14      # one TMA pass shape for both forms (else each model tunes its own)


def _model(nx, ny, prec, nshots, seed):
    om = oracle_model(nx, ny, layered(nx, ny, seed), pml=10, fs=True)
    g = gpu_model(om, prec, nshots=nshots, p=10, max_receivers=4)
    rec = np.array([[x * om.dx, 0.0] for x in (5, 11, 17, 23)])
    for s in range(nshots):
        g.set_source_receivers(s, (7 + 9 * s) * om.dx, 2 * om.dx, 25.0, 0.05, 1e3, rec)
    g.bind_seismogram(8)
    if prec == "f32":
        g.set_kernel_variant(VARIANT)   # the TMA variants differ in their rounding order
    U0s = [flatten(smooth_random_state([f.shape for f in om.zeros_state()], 40 + seed + s)) for s in range(nshots)]
    for s in range(nshots):
        g.set_state(s, U0s[s])
    return om, g, U0s


def _run(prec, column, nx=137, ny=53, nshots=3, m=12, window=0, nsteps=3):
    from paper_2401_16322_gb300.ewave import debug_set_column_kernel
    debug_set_column_kernel(column)
    try:
        om, g, U0s = _model(nx, ny, prec, nshots, 5)
        if window:
            g.set_krylov_window(window)
        for n in range(nsteps):                  # one step per call: no step graphs
            g.step("krylov", T0 + n * DT, DT, m, 1)
        g.sync()
        nv = g.vector_elems
        got = [g.unpack(g.state[s * nv:(s + 1) * nv]) for s in range(nshots)]
        out = (g.state.clone(), g.seismo.clone(), om, U0s, got)
        g.close()
        return out
    finally:
        debug_set_column_kernel(True)


def _same(a, b, prec, tol64=1e-13):
    """Bit for bit in FP32; to rounding in FP64 (relative tol64)."""
    import torch
    if prec == "f32":
        return torch.equal(a, b)
    return float((a - b).norm()) <= tol64 * float(b.norm())


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("window", [0, 3])
def test_column_kernel_equals_flat_passes_and_the_oracle(prec, window):
    s_col, seis_col, om, U0s, got = _run(prec, True, window=window)
    s_flat, seis_flat, _, _, _ = _run(prec, False, window=window)
    # the incomplete orthogonalisation of a window amplifies the FP64 rounding difference
    tol64 = 1e-10 if window else 1e-13
    d = float((s_col - s_flat).norm() / s_flat.norm())
    assert _same(s_col, s_flat, prec, tol64), d
    assert _same(seis_col, seis_flat, prec, tol64)
    if window:
        return
    for s in range(3):
        src = PointSource(om, (7 + 9 * s) * om.dx, 2 * om.dx, 25.0, 0.05, amp=1e3, p=10)
        U = unflatten(om, U0s[s])
        for n in range(3):
            U = krylov_step(om, U, src, T0 + n * DT, DT, 12)
        assert rel_l2(got[s], flatten(U)) < TOL[prec] * 3, (s, rel_l2(got[s], flatten(U)))


def test_column_kernel_with_two_chunks_per_block():
    """601 x 301 with 10 shots: 900 chunks, more than one co-resident grid holds at one chunk
    per block, so each block owns two consecutive chunks (which may belong to two shots)."""
    import torch
    s_col, seis_col, _, _, _ = _run("f32", True, nx=601, ny=301, nshots=10, m=10, nsteps=2)
    s_flat, seis_flat, _, _, _ = _run("f32", False, nx=601, ny=301, nshots=10, m=10, nsteps=2)
    assert torch.equal(s_col, s_flat)
    assert torch.equal(seis_col, seis_flat)


def test_column_kernel_in_a_batch_of_uneven_models():
    import torch
    from paper_2401_16322_gb300 import Batch
    from paper_2401_16322_gb300.ewave import debug_set_column_kernel
    states = []
    for column in (True, False):
        debug_set_column_kernel(column)
        try:
            _, g1, _ = _model(96, 41, "f32", 2, 7)
            _, g2, _ = _model(150, 70, "f32", 1, 8)
            B = Batch([g1, g2])
            B.set_kernel_variant(VARIANT)
            for n in range(2):
                B.step("krylov", T0 + n * DT, DT, 10, 1)
            B.sync()
            states.append((g1.state.clone(), g2.state.clone()))
            B.close()
            g1.close()
            g2.close()
        finally:
            debug_set_column_kernel(True)
    assert torch.equal(states[0][0], states[1][0]) and torch.equal(states[0][1], states[1][1])


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_column_kernel_in_the_exponential_adjoint(prec):
    import torch
    from paper_2401_16322_gb300.ewave import debug_set_column_kernel
    res = []
    for column in (True, False):
        debug_set_column_kernel(column)
        try:
            om, g, U0s = _model(137, 53, prec, 2, 9)
            dtype = torch.float64 if prec == "f64" else torch.float32
            nv, fe = g.vector_elems, g.layout.field_elems
            g.step("krylov", T0, DT, 12, 1)     # tunes the passes
            ck = g.state.clone()
            lam = torch.zeros(2 * nv, dtype=dtype, device="cuda")
            for s in range(2):
                g.pack(flatten(smooth_random_state([f.shape for f in om.zeros_state()], 60 + s)),
                       lam[s * nv:(s + 1) * nv])
            grad = torch.zeros(2 * fe, dtype=dtype, device="cuda")
            g.set_krylov_adjoint("exponential")
            g.adjoint_step(T0, DT, 12, ck, lam, grad, method="krylov")
            g.sync()
            res.append((lam.clone(), grad.clone()))
            g.close()
        finally:
            debug_set_column_kernel(True)
    # the Arnoldi process on dt H^T amplifies FP64 rounding differences about a thousandfold
    assert _same(res[0][0], res[1][0], prec, 1e-10) and _same(res[0][1], res[1][1], prec, 1e-10)


def test_barrier_timeout_is_reported_and_the_next_call_recovers():
    """FP64 (the plain stencil kernel, so that only the column kernel's barrier waits): with
    the wait limit at 0 the barrier gives up, the call reports EWV_ERR_TIMEOUT through the
    error word, and with the default limit restored the next step matches the oracle."""
    import torch
    from paper_2401_16322_gb300.ewave import EwaveError, debug_set_wait_limit
    om, g, U0s = _model(137, 53, "f64", 1, 11)
    g.ensure_workspace("krylov", 12)
    g.step("krylov", T0, DT, 12, 1)
    g.sync()
    try:
        debug_set_wait_limit(0)
        g.set_state(0, U0s[0])
        assert g.lib.ewv_step_krylov(g.h, T0, DT, 12, 1, None) == 0   # enqueues only
        with pytest.raises(EwaveError, match="TIMEOUT"):
            g.sync()
    finally:
        debug_set_wait_limit(1_000_000_000)
    torch.cuda.synchronize()
    g.set_state(0, U0s[0])
    g.step("krylov", T0, DT, 12, 1)
    g.sync()
    src = PointSource(om, 7 * om.dx, 2 * om.dx, 25.0, 0.05, amp=1e3, p=10)
    U = krylov_step(om, unflatten(om, U0s[0]), src, T0, DT, 12)
    assert rel_l2(g.get_state(0), flatten(U)) < TOL["f64"] * 3
    g.close()

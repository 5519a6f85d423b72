"""The allocation-free Faber entry point (ewv_faber_step_noalloc) against the regular one and
against the oracle.

Callers that cannot allocate device memory (code inside someone else's memory pool, or
environments that forbid run-time allocation) use this entry point: it needs no model handle
and keeps its work vectors in a fixed device array of the library.  This test drives it
through the C ABI on caller-owned torch tensors and checks, on two calls in a row, that it
advances the state like ewv_step_faber (within the FP32 tolerance of the other tests) and
like the FP64 oracle's Faber step, for degree 1 (the copy branch), 2 (the -2 c1 stage), 3
(an odd last degree) and 24, with and without a source.  It runs last (file name) and
passes both alone and after the rest of the suite."""
import numpy as np
import pytest

from _helpers import TOL, flatten, gpu_model, oracle_ellipse, oracle_model, rel_l2
from oracle.simulate import run
from oracle.source import PointSource
from paper_2401_16322_gb300.workloads import layered, smooth_random_state

pytestmark = pytest.mark.gpu

F_PEAK, T0, AMP, P = 25.0, 0.05, 1e3, 10


def _args(om, g, si, ell, has_source):
    from paper_2401_16322_gb300.ewave import NoallocFaberArgs
    i, j = (int(si[0]), int(si[1])) if has_source else (0, 0)
    return NoallocFaberArgs(om.nx, om.ny, g.layout.pitch, om.dx, om.order, om.pml, om.beta0,
                            int(om.free_surface), int(has_source), i, j, P, F_PEAK, T0, AMP,
                            ell[0], ell[1], ell[2])


@pytest.mark.parametrize("has_source", [True, False])
@pytest.mark.parametrize("deg", [1, 2, 3, 24])
def test_noalloc_faber_matches_regular_entry_point_and_oracle(deg, has_source):
    import torch
    from paper_2401_16322_gb300.ewave import faber_step_noalloc
    nx, ny = 137, 53
    om = oracle_model(nx, ny, layered(nx, ny, 21), pml=10, fs=True)
    g = gpu_model(om, "f32", p=P)
    sx, sy = 68 * om.dx, 2 * om.dx
    si = None
    src = None
    if has_source:
        si, _ = g.set_source_receivers(0, sx, sy, F_PEAK, T0, AMP, None)
        src = PointSource(om, sx, sy, F_PEAK, T0, amp=AMP, p=P)
    ell = oracle_ellipse(om)
    g.set_faber_ellipse(*ell)
    U0 = tuple(smooth_random_state([f.shape for f in om.zeros_state()], 31))
    g.set_state(0, flatten(U0))
    x = g.new_vector()
    g.pack(flatten(U0), x)                      # same padded initial state, caller-owned
    args = _args(om, g, si, ell, has_source)
    t, dt, per_call = 0.03, 1.2e-3, 3
    U = U0
    for call in range(2):
        t_call = t + call * per_call * dt
        g.step_faber(t_call, dt, deg, per_call)
        rc = faber_step_noalloc(args, x, g.params, t_call, dt, deg, per_call)
        assert rc == 0
        torch.cuda.synchronize()
        g.sync()
        ref = g.get_state(0)
        got = g.unpack(x)
        assert np.all(np.isfinite(got))
        assert rel_l2(got, ref) < TOL["f32"], (call, rel_l2(got, ref))
        U, _ = run(om, "faber", dt, per_call, src=src, m=deg, U0=U, t0=t_call, faber_params=ell)
        steps = (call + 1) * per_call
        assert rel_l2(got, flatten(U)) < TOL["f32"] * steps, (call, rel_l2(got, flatten(U)))
    g.close()


def test_noalloc_rejects_grids_beyond_its_array():
    import torch
    from paper_2401_16322_gb300.ewave import NOALLOC_MAX_FIELD_ELEMS, NoallocFaberArgs, faber_step_noalloc
    nx = 1024
    ny = NOALLOC_MAX_FIELD_ELEMS // nx + 1
    state = torch.zeros(16, dtype=torch.float32, device="cuda")
    c2 = torch.zeros(16, dtype=torch.float32, device="cuda")
    args = NoallocFaberArgs(nx, ny, nx, 10.0, 8, 10, 100.0, 1, 0, 0, 0, 8, 10.0, 0.27, 1.0,
                            1000.0, -0.2, -0.5)
    assert faber_step_noalloc(args, state, c2, 0.0, 1e-3, 10, 1) == -2   # BAD_SIZE_OR_ALIGNMENT
    args.ny = 4
    args.pitch = 1000                                                       # not a multiple of 32
    assert faber_step_noalloc(args, state, c2, 0.0, 1e-3, 10, 1) == -1

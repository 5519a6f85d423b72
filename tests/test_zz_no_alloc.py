"""The allocation-free Faber entry point (ewv_faber_step_noalloc) against the regular one.

Callers that cannot allocate device memory (code inside someone else's memory pool, or
environments that forbid run-time allocation) use this entry point: it needs no model handle
and keeps its work vectors in a fixed device array of the library.  This test drives it
through the C ABI on caller-owned torch tensors and checks, on two calls in a row, that it
advances the state exactly like ewv_step_faber (within the FP32 tolerance of the other tests).
It runs last (file name) and passes both alone and after the rest of the suite."""
import ctypes

import numpy as np
import pytest

from _helpers import TOL, flatten, gpu_model, oracle_ellipse, oracle_model, rel_l2
from paper_2401_16322_gb300.workloads import layered, smooth_random_state

pytestmark = pytest.mark.gpu


def _args(om, g, si, ell, p):
    from paper_2401_16322_gb300.ewave import NoallocFaberArgs
    return NoallocFaberArgs(om.nx, om.ny, g.layout.pitch, om.dx, om.order, om.pml, om.beta0,
                            int(om.free_surface), 1, int(si[0]), int(si[1]), p, 25.0, 0.05, 1e3,
                            ell[0], ell[1], ell[2])


def test_noalloc_faber_matches_regular_entry_point_on_two_calls():
    import torch
    from paper_2401_16322_gb300.ewave import faber_step_noalloc
    nx, ny, p = 137, 53, 10
    om = oracle_model(nx, ny, layered(nx, ny, 21), pml=10, fs=True)
    g = gpu_model(om, "f32", p=p)
    si, _ = g.set_source_receivers(0, 68 * om.dx, 2 * om.dx, 25.0, 0.05, 1e3, None)
    ell = oracle_ellipse(om)
    g.set_faber_ellipse(*ell)
    U0 = tuple(smooth_random_state([f.shape for f in om.zeros_state()], 31))
    g.set_state(0, flatten(U0))
    x = g.new_vector()
    g.pack(flatten(U0), x)                      # same padded initial state, caller-owned
    args = _args(om, g, si, ell, p)
    t, dt, deg = 0.03, 1.2e-3, 24
    for call in range(2):
        t_call = t + call * 3 * dt
        g.step_faber(t_call, dt, deg, 3)
        rc = faber_step_noalloc(args, x, g.params, t_call, dt, deg, 3)
        assert rc == 0
        torch.cuda.synchronize()
        ref = g.get_state(0)
        got = g.unpack(x)
        assert np.all(np.isfinite(got))
        assert rel_l2(got, ref) < TOL["f32"], (call, rel_l2(got, ref))


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

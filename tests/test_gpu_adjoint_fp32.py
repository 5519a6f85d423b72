"""FP32 adjoint steps through the persistent TMA passes (forward recompute, gradient and the
transposed pass H^T on the column-pair consumers; for Krylov, the adjoint of the step's
exponential with both Arnoldi processes on the TMA passes and split dots) against the
oracle's adjoint steps, on
grids that span several 64 x 18 tiles with ragged tails, with and without the free surface
(whose transposed rows, 0..8, take the kernel's scalar path) and at both orders."""
import numpy as np
import pytest

from _helpers import flatten, rel_l2
from oracle.adjoint import faber_adjoint_step, hork_adjoint_step, krylov_adjoint_step
from oracle.faber import ellipse_params
from oracle.model import Model as OModel
from oracle.model import default_beta0
from oracle.source import PointSource
from paper_2401_16322_gb300.workloads import layered, random_state, smooth_random_state

pytestmark = pytest.mark.gpu

CASES = [
    # (nx, ny, order, fs, pml)
    (137, 53, 8, True, 12),
    (70, 39, 8, False, 9),
    (101, 41, 4, False, 20),
    (66, 20, 8, True, 0),
]
DX = 10.0


@pytest.mark.parametrize("method,m", [("faber", 6), ("hork", 5), ("krylov", 8)])
@pytest.mark.parametrize("nx,ny,order,fs,pml", CASES)
def test_fp32_adjoint_step_matches_oracle(method, m, nx, ny, order, fs, pml):
    import torch
    from paper_2401_16322_gb300 import Model
    c = layered(nx, ny, 12, vmin=1500, vmax=3000)
    beta0 = default_beta0(3000.0, pml, DX)
    om = OModel(nx, ny, DX, order, pml, beta0, fs, c)
    ell = ellipse_params(3000.0, beta0, DX, order, free_surface=fs)
    sxs = [(nx // 3) * DX, (2 * nx // 3) * DX]
    g = Model(nx, ny, DX, order, pml, beta0, fs, precision="f32", nshots=2, p=8)
    g.set_velocity(c)
    for k, sx in enumerate(sxs):
        g.set_source_receivers(k, sx, 2 * DX, 30.0, 0.04, 1e3, np.zeros((0, 2)))
    g.set_faber_ellipse(*ell)
    dt, t = 1.2e-3, 0.02
    g.step(method, t, dt, m, 1)          # a forward step: the stencil passes are tuned
    nv, fe = g.vector_elems, g.layout.field_elems
    Us = [flatten(smooth_random_state([f.shape for f in om.zeros_state()], 50 + k)) for k in range(2)]
    ybars = [random_state([(om.n,)], 60 + k)[0] for k in range(2)]
    ck = torch.zeros(2 * nv, dtype=torch.float32, device="cuda")
    lam = torch.zeros(2 * nv, dtype=torch.float32, device="cuda")
    for k in range(2):
        g.pack(Us[k], ck[k * nv:(k + 1) * nv])
        g.pack(ybars[k], lam[k * nv:(k + 1) * nv])
    grad = torch.zeros(2 * fe, dtype=torch.float32, device="cuda")
    if method == "krylov":
        g.set_krylov_adjoint("exponential")
    g.adjoint_step(t, dt, m, ck, lam, grad, method=method)
    g.sync()
    for k, sx in enumerate(sxs):
        src = PointSource(om, sx, 2 * DX, 30.0, 0.04, amp=1e3, p=8)
        if method == "faber":
            Ub, gr = faber_adjoint_step(om, Us[k], ybars[k], src, t, dt, m, ell)
        elif method == "krylov":
            Ub, gr = krylov_adjoint_step(om, Us[k], ybars[k], src, t, dt, m)
        else:
            Ub, gr = hork_adjoint_step(om, Us[k], ybars[k], src, t, dt, m)
        got = g.unpack(lam[k * nv:(k + 1) * nv])
        assert rel_l2(got, Ub) < 3e-5, (k, rel_l2(got, Ub))
        g_got = grad[k * fe:(k + 1) * fe].view(ny, g.layout.pitch)[:, :nx].double().cpu().numpy()
        assert rel_l2(g_got, gr.reshape(ny, nx)) < 3e-5, (k, rel_l2(g_got, gr.reshape(ny, nx)))
    g.close()

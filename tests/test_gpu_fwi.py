"""GPU FWI gradient (m = c^2) through the discrete adjoint of the Faber step: the adjoint
dot-product identity on the GPU, the oracle's gradient, central finite differences,
checkpointing, FP32, and the torch.autograd path."""
import numpy as np
import pytest

from oracle.adjoint import checkpoint_stride as o_stride
from oracle.adjoint import faber_forward, fwi_gradient, misfit
from oracle.faber import ellipse_params
from oracle.model import Model as OModel
from oracle.model import default_beta0, flatten
from oracle.simulate import receiver_nodes, rel_l2
from oracle.source import PointSource
from paper_2401_16322_gb300.workloads import layered, random_state, smooth_random_state

pytestmark = pytest.mark.gpu

NX, NY, DX, PML = 30, 20, 10.0, 5
DT, NSTEPS, DEG = 2e-3, 14, 12
SX = (8 * DX, 21 * DX)
REC = np.array([[x * DX, 0.0] for x in range(3, NX - 3, 4)])


def _setup():
    c_true = layered(NX, NY, 31, vmin=1500, vmax=3000)
    c0 = np.full((NY, NX), float(c_true.mean()))
    beta0 = default_beta0(3000.0, PML, DX)
    ell = ellipse_params(3000.0, beta0, DX, 8, free_surface=True)
    return c_true, c0, beta0, ell


def _oshots(om):
    return [(PointSource(om, sx, 2 * DX, 30.0, 0.04, amp=1e3, p=10), receiver_nodes(om, REC)) for sx in SX]


def _gpu(c, beta0, ell, prec, sources=True):
    from paper_2401_16322_gb300 import Model
    g = Model(NX, NY, DX, 8, PML, beta0, True, precision=prec, nshots=2, p=10, max_receivers=len(REC))
    g.set_velocity(c)
    if sources:
        for k, sx in enumerate(SX):
            g.set_source_receivers(k, sx, 2 * DX, 30.0, 0.04, 1e3, REC)
    g.set_faber_ellipse(*ell)
    return g


def _d_obs():
    c_true, c0, beta0, ell = _setup()
    om = OModel(NX, NY, DX, 8, PML, beta0, True, c_true)
    return faber_forward(om, _oshots(om), DT, NSTEPS, DEG, ell)[1]


def _gpu_grad(prec, budget=None, variant=None):
    import torch
    from paper_2401_16322_gb300.fwi import FaberFWI
    c_true, c0, beta0, ell = _setup()
    g = _gpu(c0, beta0, ell, prec)
    if variant is not None:
        g.set_kernel_variant(variant)
    fwi = FaberFWI(g, DT, DEG, NSTEPS, len(REC), budget=budget)
    seis = fwi.forward(c0 ** 2)
    d = torch.tensor(np.array(_d_obs()), dtype=seis.dtype, device=seis.device)
    grad = fwi.backward(seis - d)
    J = 0.5 * float(((seis - d) ** 2).sum())
    return J, grad.double().cpu().numpy(), fwi


def test_adjoint_step_dot_product_identity_gpu():
    """<A dU, ybar> = <dU, A^T ybar> for one Faber step's linear part (no source)."""
    import torch
    c_true, c0, beta0, ell = _setup()
    g = _gpu(c_true, beta0, ell, "f64", sources=False)
    om = OModel(NX, NY, DX, 8, PML, beta0, True, c_true)
    dU, yb = (random_state([(om.n,)], s)[0] for s in (3, 4))
    g.set_state(0, dU)
    g.set_state(1, dU)
    g.step_faber(0.0, DT, DEG, 1)
    AdU = g.get_state(0)
    ck = torch.zeros_like(g.state)
    lam = g.new_vector().repeat(2)
    nv = g.vector_elems
    g.pack(yb, lam[:nv])
    grad = torch.zeros(2 * g.layout.field_elems, dtype=torch.float64, device="cuda")
    g.adjoint_step(0.0, DT, DEG, ck, lam, grad)
    q0 = g.unpack(lam[:nv])
    lhs, rhs = float(np.dot(AdU, yb)), float(np.dot(dU, q0))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_gpu_gradient_matches_oracle_fp64():
    c_true, c0, beta0, ell = _setup()
    om = OModel(NX, NY, DX, 8, PML, beta0, True, c0)
    J_o, g_o = fwi_gradient(om, _oshots(om), _d_obs(), DT, NSTEPS, DEG, ell)
    J_g, g_g, _ = _gpu_grad("f64")
    assert abs(J_g - J_o) <= 1e-11 * J_o
    assert rel_l2(g_g, g_o) < 1e-10


def test_gpu_gradient_central_differences_fp64():
    """Directional derivative of the GPU misfit by central differences, relative 1e-3."""
    import torch
    from paper_2401_16322_gb300.fwi import FaberFWI
    c_true, c0, beta0, ell = _setup()
    J0, grad, fwi = _gpu_grad("f64")
    d = torch.tensor(np.array(_d_obs()), dtype=torch.float64, device="cuda")
    c2 = c0 ** 2
    for seed in (5, 6, 7):
        dm = smooth_random_state([(NY, NX)], seed, sigma_cells=2.0)[0] * 0.01 * c2
        eps = 1e-4
        Jp = 0.5 * float(((fwi.forward(c2 + eps * dm) - d) ** 2).sum())
        Jm = 0.5 * float(((fwi.forward(c2 - eps * dm) - d) ** 2).sum())
        fd = (Jp - Jm) / (2 * eps)
        an = float(np.sum(grad * dm))
        assert abs(fd - an) <= 1e-3 * abs(fd), (seed, fd, an)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_checkpointing_reproduces_full_storage(prec):
    """Storing every 4th state (segments recomputed) gives the same gradient bit for bit.  The
    two models are pinned to one stencil-pass variant: models tuned separately may pick
    different variants, which agree to rounding only."""
    _, g_full, fwi1 = _gpu_grad(prec, variant=0)
    _, g_ck, fwi4 = _gpu_grad(prec, budget=4, variant=0)
    assert fwi1.stride == 1 and fwi4.stride == o_stride(NSTEPS, 4) == 4
    assert np.array_equal(g_full, g_ck)


def test_fp32_gradient_against_fp64_oracle():
    c_true, c0, beta0, ell = _setup()
    om = OModel(NX, NY, DX, 8, PML, beta0, True, c0)
    _, g_o = fwi_gradient(om, _oshots(om), _d_obs(), DT, NSTEPS, DEG, ell)
    _, g32, _ = _gpu_grad("f32")
    assert rel_l2(g32, g_o) < 1e-3


def test_autograd_function_gives_the_adjoint_gradient():
    import torch
    from paper_2401_16322_gb300.fwi import FaberFWI, seismogram_fn
    c_true, c0, beta0, ell = _setup()
    g = _gpu(c0, beta0, ell, "f64")
    fwi = FaberFWI(g, DT, DEG, NSTEPS, len(REC))
    m = torch.tensor(c0 ** 2, dtype=torch.float64, requires_grad=True)
    d = torch.tensor(np.array(_d_obs()), dtype=torch.float64, device="cuda")
    seis = seismogram_fn().apply(m, fwi)
    loss = 0.5 * ((seis - d) ** 2).sum()
    loss.backward()
    _, g_ref, _ = _gpu_grad("f64")
    assert np.allclose(m.grad.cpu().numpy(), g_ref, rtol=1e-12, atol=0)


def test_hork_gradient_matches_oracle_and_differences():
    """HORK (8 stages, dt 0.5 ms): GPU adjoint gradient = oracle (FP64), and central
    differences of the GPU misfit along a seeded direction."""
    import torch
    from paper_2401_16322_gb300.fwi import FaberFWI
    c_true, c0, beta0, ell = _setup()
    dt, deg = 5e-4, 8
    om_t = OModel(NX, NY, DX, 8, PML, beta0, True, c_true)
    d_obs = faber_forward(om_t, _oshots(om_t), dt, NSTEPS, deg, ell, method="hork")[1]
    om = OModel(NX, NY, DX, 8, PML, beta0, True, c0)
    J_o, g_o = fwi_gradient(om, _oshots(om), d_obs, dt, NSTEPS, deg, ell, method="hork")
    g = _gpu(c0, beta0, ell, "f64")
    fwi = FaberFWI(g, dt, deg, NSTEPS, len(REC), method="hork")
    d = torch.tensor(np.array(d_obs), dtype=torch.float64, device="cuda")
    seis = fwi.forward(c0 ** 2)
    grad = fwi.backward(seis - d).double().cpu().numpy()
    assert rel_l2(grad, g_o) < 1e-10
    dm = smooth_random_state([(NY, NX)], 9, sigma_cells=2.0)[0] * 0.01 * c0 ** 2
    eps = 1e-4
    Jp = 0.5 * float(((fwi.forward(c0 ** 2 + eps * dm) - d) ** 2).sum())
    Jm = 0.5 * float(((fwi.forward(c0 ** 2 - eps * dm) - d) ** 2).sum())
    fd = (Jp - Jm) / (2 * eps)
    assert abs(fd - float(np.sum(grad * dm))) <= 1e-3 * abs(fd)


def test_checkpoint_stride_bit_exact():
    from paper_2401_16322_gb300.ewave import checkpoint_stride
    for n in range(0, 60):
        for b in range(1, 25):
            assert checkpoint_stride(n, b) == o_stride(n, b)


@pytest.mark.parametrize("budget", [None, 4])
def test_krylov_gradient_matches_oracle_and_differences(budget):
    """Krylov (m = 12, dt 1 ms), the adjoint of the step's exponential (the library's
    EWV_KRYLOV_ADJOINT_EXPONENTIAL option): the linearised adjoint gradient on the GPU equals the oracle's
    (FP64), with and without checkpoint segments, and agrees with central differences of the
    GPU Krylov misfit to the step's time accuracy (1e-3)."""
    import torch
    from paper_2401_16322_gb300.fwi import FaberFWI
    c_true, c0, beta0, ell = _setup()
    dt, m, nsteps = 1e-3, 12, 10
    om_t = OModel(NX, NY, DX, 8, PML, beta0, True, c_true)
    d_obs = faber_forward(om_t, _oshots(om_t), dt, nsteps, m, ell, method="krylov")[1]
    om = OModel(NX, NY, DX, 8, PML, beta0, True, c0)
    J_o, g_o = fwi_gradient(om, _oshots(om), d_obs, dt, nsteps, m, ell, method="krylov")
    g = _gpu(c0, beta0, ell, "f64")
    g.set_krylov_adjoint("exponential")
    fwi = FaberFWI(g, dt, m, nsteps, len(REC), budget=budget, method="krylov")
    d = torch.tensor(np.array(d_obs), dtype=torch.float64, device="cuda")
    seis = fwi.forward(c0 ** 2)
    assert abs(0.5 * float(((seis - d) ** 2).sum()) - J_o) <= 1e-9 * J_o
    grad = fwi.backward(seis - d).double().cpu().numpy()
    assert rel_l2(grad, g_o) < 1e-9
    dm = smooth_random_state([(NY, NX)], 9, sigma_cells=2.0)[0] * 0.01 * c0 ** 2
    eps = 1e-4
    Jp = 0.5 * float(((fwi.forward(c0 ** 2 + eps * dm) - d) ** 2).sum())
    Jm = 0.5 * float(((fwi.forward(c0 ** 2 - eps * dm) - d) ** 2).sum())
    fd = (Jp - Jm) / (2 * eps)
    assert abs(fd - float(np.sum(grad * dm))) <= 1e-3 * abs(fd)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_krylov_dense_step_and_adjoint(prec, tol):
    """ewv_step_krylov_dense leaves the state ewv_step_krylov leaves (bit for bit: the same
    passes) and writes the oracle's four dense states (Sec. 3.2 dense output at the
    Gauss-Legendre nodes); the adjoint from those states equals the exponential adjoint that
    recomputes the forward Arnoldi from the checkpoint, and the oracle's.  In FP64 the adjoint
    is held to 1e-10, not 1e-12: the Arnoldi process on dt H^T amplifies rounding-order
    differences about a thousandfold here (perturbing the oracle's cotangent by one part in
    1e16 moves its result by up to 3e-13)."""
    import torch
    from oracle.adjoint import krylov_adjoint_step, krylov_dense_states
    c_true, c0, beta0, ell = _setup()
    om = OModel(NX, NY, DX, 8, PML, beta0, True, c_true)
    g = _gpu(c_true, beta0, ell, prec)
    g.bind_seismogram(4)
    dtype = torch.float64 if prec == "f64" else torch.float32
    ns, nv, fe = 2, g.vector_elems, g.layout.field_elems
    t, dt, m = 0.02, 2e-3, 12
    Us = [flatten(smooth_random_state([f.shape for f in om.zeros_state()], 70 + k)) for k in range(ns)]
    ybars = [random_state([(om.n,)], 80 + k)[0] for k in range(ns)]
    u0 = torch.zeros(ns * nv, dtype=dtype, device="cuda")
    y0 = torch.zeros(ns * nv, dtype=dtype, device="cuda")
    for k in range(ns):
        g.pack(Us[k], u0[k * nv:(k + 1) * nv])
        g.pack(ybars[k], y0[k * nv:(k + 1) * nv])
    g.step_krylov(t, dt, m)                  # tunes the passes before the comparison
    g.state.copy_(u0)
    g.step_krylov(t, dt, m)
    ref = g.state.clone()
    xd = torch.zeros(4 * ns * nv, dtype=dtype, device="cuda")
    g.state.copy_(u0)
    g.step_krylov_dense(t, dt, m, xd)
    g.sync()
    assert torch.equal(g.state[:ns * nv], ref[:ns * nv])
    lam_r, lam_d = y0.clone(), y0.clone()
    grad_r = torch.zeros(ns * fe, dtype=dtype, device="cuda")
    grad_d = torch.zeros(ns * fe, dtype=dtype, device="cuda")
    g.set_krylov_adjoint("exponential")
    g.adjoint_step(t, dt, m, u0, lam_r, grad_r, method="krylov")
    g.adjoint_step_krylov_dense(t, dt, m, xd, lam_d, grad_d)
    g.sync()
    assert float((lam_d - lam_r).norm() / lam_r.norm()) < 1e-6 * (1e-6 if prec == "f64" else 1.0)
    assert float((grad_d - grad_r).norm() / grad_r.norm()) < 1e-6 * (1e-6 if prec == "f64" else 1.0)
    for k, sx in enumerate(SX):
        src = PointSource(om, sx, 2 * DX, 30.0, 0.04, amp=1e3, p=10)
        want = krylov_dense_states(om, Us[k], src, t, dt, m)
        for q in range(4):
            got = g.unpack(xd[(q * ns + k) * nv:(q * ns + k + 1) * nv])
            assert rel_l2(got, want[q]) < tol, (k, q, rel_l2(got, want[q]))
        Ub, gr = krylov_adjoint_step(om, Us[k], ybars[k], src, t, dt, m)
        tol_adj = 1e-10 if prec == "f64" else tol
        e_lam = rel_l2(g.unpack(lam_d[k * nv:(k + 1) * nv]), Ub)
        g_got = grad_d[k * fe:(k + 1) * fe].view(NY, g.layout.pitch)[:, :NX].double().cpu().numpy()
        e_grad = rel_l2(g_got, gr.reshape(NY, NX))
        assert e_lam < tol_adj and e_grad < tol_adj, (k, e_lam, e_grad)
    g.close()


@pytest.mark.parametrize("budget", [None, 4])
def test_krylov_dense_state_gradient_matches_oracle(budget):
    """FWI gradient with the forward's dense states (no forward Arnoldi in the adjoint):
    every step's states stored, or a segment's recomputed from its checkpoint; equals the
    oracle's exponential-adjoint gradient (FP64) and the recomputing path's."""
    import torch
    from paper_2401_16322_gb300.fwi import FaberFWI
    c_true, c0, beta0, ell = _setup()
    dt, m, nsteps = 1e-3, 12, 10
    om_t = OModel(NX, NY, DX, 8, PML, beta0, True, c_true)
    d_obs = faber_forward(om_t, _oshots(om_t), dt, nsteps, m, ell, method="krylov")[1]
    om = OModel(NX, NY, DX, 8, PML, beta0, True, c0)
    J_o, g_o = fwi_gradient(om, _oshots(om), d_obs, dt, nsteps, m, ell, method="krylov")
    g = _gpu(c0, beta0, ell, "f64")
    g.set_krylov_adjoint("exponential")
    d = torch.tensor(np.array(d_obs), dtype=torch.float64, device="cuda")
    fwi = FaberFWI(g, dt, m, nsteps, len(REC), budget=budget, method="krylov", dense_states=True)
    seis = fwi.forward(c0 ** 2)
    assert abs(0.5 * float(((seis - d) ** 2).sum()) - J_o) <= 1e-9 * J_o
    grad = fwi.backward(seis - d).double().cpu().numpy()
    assert rel_l2(grad, g_o) < 1e-9
    ref = FaberFWI(g, dt, m, nsteps, len(REC), budget=budget, method="krylov")
    grad_r = ref.backward(ref.forward(c0 ** 2) - d).double().cpu().numpy()
    assert rel_l2(grad, grad_r) < 1e-12
    if budget is None:
        assert fwi.ckpt.numel() == 0 and fwi.xd.shape[0] == nsteps
    g.close()


# ---------------------------------------------------------------- leap-frog adjoint
LF_DT, LF_NSTEPS = 1e-3, 30


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 3e-5)])
def test_leapfrog_adjoint_step_is_the_oracle_transpose(prec, tol):
    """One leap-frog adjoint step on the GPU (two shots) against the transpose of the
    oracle's assembled step matrix (oracle/leapfrog_adjoint.py) applied to a random cotangent
    of (u, u_prev, w, w_prev), and the gradient increment s G(u^n, w^n) lambda_u.  The
    cotangent buffer holds 2 nshots vectors: level n of every shot, then w_prev of every shot.
    FP32 runs the gradient and transposed passes on the persistent TMA kernels (a forward
    step first tunes them)."""
    import torch
    from oracle import leapfrog_adjoint as LA
    c_true, c0, beta0, ell = _setup()
    om = OModel(NX, NY, DX, 8, PML, beta0, True, c_true)
    g = _gpu(c_true, beta0, ell, prec, sources=False)
    if prec == "f32":
        g.step_faber(0.0, LF_DT, 2, 1)
    dtype = torch.float64 if prec == "f64" else torch.float32
    ns, nv, fe = g.nshots, g.vector_elems, g.layout.field_elems
    nu = NX * NY
    nwx, nwy = NY * (NX - 1), (NY - 1) * NX
    A, s = LA.step_matrix(om, LF_DT)
    ck = torch.zeros(ns * nv, dtype=dtype, device="cuda")
    adj = torch.zeros(2 * ns * nv, dtype=dtype, device="cuda")
    grad = torch.zeros(ns * fe, dtype=dtype, device="cuda")
    lams, states = [], []
    for k in range(ns):
        lam = random_state([(nu,), (nu,), (nwx,), (nwy,), (nwx,), (nwy,)], 13 + k)
        st = smooth_random_state([(nu,), (nwx,), (nwy,)], 14 + k)
        g.pack(np.concatenate([st[0], np.zeros(nu), st[1], st[2]]), ck[k * nv:(k + 1) * nv])
        g.pack(np.concatenate(lam[:4]), adj[k * nv:(k + 1) * nv])
        g.pack(np.concatenate([np.zeros(2 * nu), lam[4], lam[5]]), adj[(ns + k) * nv:(ns + k + 1) * nv])
        lams.append(lam)
        states.append(st)
    g.adjoint_step(0.0, LF_DT, 0, ck, adj, grad, method="leapfrog")
    g.sync()
    for k in range(ns):
        a0 = g.unpack(adj[k * nv:(k + 1) * nv])
        a1 = g.unpack(adj[(ns + k) * nv:(ns + k + 1) * nv])
        got = np.concatenate([a0[:nu], a0[nu:2 * nu], a0[2 * nu:], a1[2 * nu:]])
        ref = A.T @ np.concatenate(lams[k])
        assert rel_l2(got, ref) < tol, k
        u, wx, wy = states[k]
        G = LA._G(om, u.reshape(NY, NX), wx.reshape(NY, NX - 1), wy.reshape(NY - 1, NX)).ravel()
        g_ref = (s * G * lams[k][0]).reshape(NY, NX)
        g_got = grad[k * fe:(k + 1) * fe].view(NY, g.layout.pitch)[:, :NX].double().cpu().numpy()
        assert rel_l2(g_got, g_ref) < tol, k


def _lf_shots(om):
    return [(PointSource(om, sx, 2 * DX, 30.0, 0.04, amp=1e3, p=10), receiver_nodes(om, REC)) for sx in SX]


@pytest.mark.parametrize("variant", ["averaged", "difference"])
def test_leapfrog_gradient_matches_oracle_checkpointing_and_differences(variant):
    """The FWI gradient through leap-frog steps (two shots, 30 steps of 1 ms, FP64): GPU =
    oracle's discrete adjoint (1e-10), checkpoints every 4th step (two time levels each,
    segments recomputed) reproduce full storage bit for bit, and central differences of the
    GPU misfit agree (1e-3).  The difference form is the same scheme and has the same
    adjoint."""
    import torch
    from oracle import leapfrog_adjoint as LA
    from paper_2401_16322_gb300.ewave import LEAPFROG_AVERAGED, LEAPFROG_DIFFERENCE
    from paper_2401_16322_gb300.fwi import FaberFWI
    c_true, c0, beta0, ell = _setup()
    om_t = OModel(NX, NY, DX, 8, PML, beta0, True, c_true)
    d_obs = LA.forward(om_t, _lf_shots(om_t), LF_DT, LF_NSTEPS)[1]
    om = OModel(NX, NY, DX, 8, PML, beta0, True, c0)
    J_o, g_o = LA.fwi_gradient(om, _lf_shots(om), d_obs, LF_DT, LF_NSTEPS)
    d = torch.tensor(np.array(d_obs), dtype=torch.float64, device="cuda")
    grads = []
    for budget in (None, 8):
        g = _gpu(c0, beta0, ell, "f64")
        g.set_leapfrog_variant(LEAPFROG_DIFFERENCE if variant == "difference" else LEAPFROG_AVERAGED)
        fwi = FaberFWI(g, LF_DT, 0, LF_NSTEPS, len(REC), budget=budget, method="leapfrog")
        seis = fwi.forward(c0 ** 2)
        assert abs(0.5 * float(((seis - d) ** 2).sum()) - J_o) <= 1e-9 * J_o
        grads.append(fwi.backward(seis - d).double().cpu().numpy())
    assert fwi.stride == 4
    assert rel_l2(grads[0], g_o) < 1e-10
    assert np.array_equal(grads[0], grads[1])
    dm = smooth_random_state([(NY, NX)], 9, sigma_cells=2.0)[0] * 0.01 * c0 ** 2
    eps = 1e-4
    Jp = 0.5 * float(((fwi.forward(c0 ** 2 + eps * dm) - d) ** 2).sum())
    Jm = 0.5 * float(((fwi.forward(c0 ** 2 - eps * dm) - d) ** 2).sum())
    fd = (Jp - Jm) / (2 * eps)
    assert abs(fd - float(np.sum(grads[0] * dm))) <= 1e-3 * abs(fd)


def test_leapfrog_adjoint_rejects_the_literal_variant():
    import torch
    from paper_2401_16322_gb300.ewave import LEAPFROG_LITERAL, EwaveError
    c_true, c0, beta0, ell = _setup()
    g = _gpu(c_true, beta0, ell, "f64", sources=False)
    g.set_leapfrog_variant(LEAPFROG_LITERAL)
    ns, nv = g.nshots, g.vector_elems
    ck = torch.zeros(ns * nv, dtype=torch.float64, device="cuda")
    adj = torch.zeros(2 * ns * nv, dtype=torch.float64, device="cuda")
    grad = torch.zeros(ns * g.layout.field_elems, dtype=torch.float64, device="cuda")
    with pytest.raises(EwaveError, match="UNSUPPORTED"):
        g.adjoint_step(0.0, LF_DT, 0, ck, adj, grad, method="leapfrog")


# ---------------------------------------------------------------- exact Krylov adjoint
@pytest.mark.parametrize("mm,window,at_rest", [(1, 0, False), (6, 0, False), (12, 0, False),
                                               (12, 3, False), (20, 0, True)])
def test_krylov_exact_adjoint_step_matches_oracle(mm, window, at_rest):
    """One exact Krylov adjoint step on the GPU (FP64, two shots with their sources) against the
    oracle's reverse mode through the same step (oracle/krylov_adjoint.py): the cotangent of
    U^{n-1} and the gradient increment, 1e-10.  Covers m = 1, full and windowed Gram-Schmidt,
    and a step from rest (U = 0: eta fixed at 1, the basis breaks down after the tail's
    dimension, so the reverse sweep starts at m_eff < m)."""
    import torch
    from oracle.krylov_adjoint import krylov_exact_adjoint_step
    c_true, c0, beta0, ell = _setup()
    om = OModel(NX, NY, DX, 8, PML, beta0, True, c0)
    g = _gpu(c0, beta0, ell, "f64")
    g.set_krylov_window(window)
    dt, t = 1.5e-3, 0.03
    nv, fe = g.vector_elems, g.layout.field_elems
    Us = [np.zeros(om.n) if at_rest else flatten(smooth_random_state([f.shape for f in om.zeros_state()], 30 + k))
          for k in range(2)]
    ybars = [random_state([(om.n,)], 40 + k)[0] for k in range(2)]
    ck = torch.zeros(2 * nv, dtype=torch.float64, device="cuda")
    lam = torch.zeros(2 * nv, dtype=torch.float64, device="cuda")
    for k in range(2):
        g.pack(Us[k], ck[k * nv:(k + 1) * nv])
        g.pack(ybars[k], lam[k * nv:(k + 1) * nv])
    grad = torch.zeros(2 * fe, dtype=torch.float64, device="cuda")
    g.adjoint_step(t, dt, mm, ck, lam, grad, method="krylov")
    g.sync()
    for k, (src, _) in enumerate(_oshots(om)):
        Ub, gr = krylov_exact_adjoint_step(om, Us[k], ybars[k], src, t, dt, mm,
                                           window=window or None)
        assert rel_l2(g.unpack(lam[k * nv:(k + 1) * nv]), Ub) < 1e-10, k
        g_got = grad[k * fe:(k + 1) * fe].view(NY, g.layout.pitch)[:, :NX].cpu().numpy()
        assert rel_l2(g_got, gr.reshape(NY, NX)) < 1e-9, k
    g.close()


@pytest.mark.parametrize("budget", [None, 4])
def test_krylov_exact_gradient_at_the_benchmark_setting(budget):
    """The FWI gradient through Krylov steps of dimension 20 at 8 x the leap-frog step (the
    setting bench.py times), FP64: the GPU's exact discrete adjoint equals the oracle's
    (1e-9), checkpoint segments reproduce full storage, and central differences of the GPU
    misfit agree to 1e-3 -- the gradient of the misfit of the computed Krylov steps."""
    import torch
    from oracle.krylov_adjoint import krylov_exact_fwi_gradient
    from paper_2401_16322_gb300.fwi import FaberFWI
    from paper_2401_16322_gb300.tts import leapfrog_step
    c_true, c0, beta0, ell = _setup()
    mm, nsteps = 20, 8
    dt = 8.0 * leapfrog_step(3000.0, DX)
    om_t = OModel(NX, NY, DX, 8, PML, beta0, True, c_true)
    d_obs = faber_forward(om_t, _oshots(om_t), dt, nsteps, mm, ell, method="krylov")[1]
    om = OModel(NX, NY, DX, 8, PML, beta0, True, c0)
    J_o, g_o = krylov_exact_fwi_gradient(om, _oshots(om), d_obs, dt, nsteps, mm)
    g = _gpu(c0, beta0, ell, "f64")
    fwi = FaberFWI(g, dt, mm, nsteps, len(REC), budget=budget, method="krylov")
    d = torch.tensor(np.array(d_obs), dtype=torch.float64, device="cuda")
    seis = fwi.forward(c0 ** 2)
    assert abs(0.5 * float(((seis - d) ** 2).sum()) - J_o) <= 1e-9 * J_o
    grad = fwi.backward(seis - d).double().cpu().numpy()
    assert rel_l2(grad, g_o) < 1e-9          # measured 3.0e-10: 8 steps of dimension 20
    dm = smooth_random_state([(NY, NX)], 9, sigma_cells=2.0)[0] * 0.01 * c0 ** 2
    eps = 1e-4
    Jp = 0.5 * float(((fwi.forward(c0 ** 2 + eps * dm) - d) ** 2).sum())
    Jm = 0.5 * float(((fwi.forward(c0 ** 2 - eps * dm) - d) ** 2).sum())
    fd = (Jp - Jm) / (2 * eps)
    assert abs(fd - float(np.sum(grad * dm))) <= 1e-3 * abs(fd)


def _fwi_workload_fd(method, m, k, prec, eps, adjoint=None):
    """(relative FD mismatch, gradient) of the FWI gradient on the 16-shot FWI workload
    (401 x 201, 200 receivers, T = 1.5 s) at step k x the leap-frog step."""
    import torch
    from paper_2401_16322_gb300.fwi import FaberFWI
    from paper_2401_16322_gb300.tts import build_models, common_ellipse, leapfrog_step
    from paper_2401_16322_gb300.workloads import config_fwi, smooth_gradient_with_anomalies
    w = config_fwi()
    c_max = float(w.c.max()) * 1.05
    dt = k * leapfrog_step(c_max, w.dx, w.order)
    nsteps = int(round(w.T / dt))
    c_init = smooth_gradient_with_anomalies(w.nx, w.ny, 0, dx=w.dx, amps=())
    dm = smooth_random_state([(w.ny, w.nx)], 5, sigma_cells=8.0)[0] * 0.01 * c_init ** 2
    md = build_models([w], prec, p=12, c_max=c_max)[0]
    common_ellipse([md], c_max)
    if adjoint:
        md.set_krylov_adjoint(adjoint)
    fwi = FaberFWI(md, dt, m, nsteps, len(w.shots[0].rec), method=method)
    d_obs = fwi.forward(w.c ** 2).double()
    seis = fwi.forward(c_init ** 2).double()
    grad = fwi.backward(seis - d_obs).double().cpu().numpy()

    def J(c2):
        return 0.5 * float(((fwi.forward(c2).double() - d_obs) ** 2).sum())

    fd = (J(c_init ** 2 + eps * dm) - J(c_init ** 2 - eps * dm)) / (2 * eps)
    md.close()
    torch.cuda.empty_cache()
    return abs(fd - float(np.sum(grad * dm))) / abs(fd), grad


def test_krylov_gradient_central_differences_on_the_fwi_workload():
    """The 16-shot FWI workload itself: central differences of the GPU misfit against the
    adjoint gradient.
    - Krylov 20 at 4 x the leap-frog step, exact discrete adjoint, FP64: 1e-3 (measured
      2.0e-5, the O(eps^2) term of the difference).
    - Krylov 20 at 8 x (the benchmark setting), FP64: the exact adjoint of that step is
      ill-conditioned over 148 steps (its cotangent grows by ~1e85 while the source is still
      silent), so the FWI runs take the adjoint of the step's exponential, which agrees with
      the differences of the computed Krylov misfit to the step's own accuracy: 2e-3
      (measured 8.9e-4).
    - FP32 at 8 x: the gradient is within 1e-3 of the FP64 one (measured 2.7e-4) and agrees
      with FP32 differences to 1e-2 (measured 2.1e-3; FP32 rounding of the misfit)."""
    err4, _ = _fwi_workload_fd("krylov", 20, 4.0, "f64", 1e-3)
    assert err4 <= 1e-3, err4
    err8, g64 = _fwi_workload_fd("krylov", 20, 8.0, "f64", 1e-3, adjoint="exponential")
    assert err8 <= 2e-3, err8
    err32, g32 = _fwi_workload_fd("krylov", 20, 8.0, "f32", 1e-2, adjoint="exponential")
    assert rel_l2(g32, g64) < 1e-3, rel_l2(g32, g64)
    assert err32 <= 1e-2, err32


def test_hork_gradient_central_differences_on_the_fwi_workload():
    """The same workload with Horner HORK 20 at 4 x (the FWI gradient bench.py times): the exact
    discrete adjoint of the linear step agrees with FP64 central differences to 1e-4 (measured
    2.0e-5), and the FP32 gradient is within 1e-3 of the FP64 one (measured 1.5e-4)."""
    err, g64 = _fwi_workload_fd("hork", 20, 4.0, "f64", 1e-3)
    assert err <= 1e-4, err
    _, g32 = _fwi_workload_fd("hork", 20, 4.0, "f32", 1e-2)
    assert rel_l2(g32, g64) < 1e-3, rel_l2(g32, g64)

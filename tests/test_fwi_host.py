"""Host logic of the FWI driver (paper_2401_16322_gb300/fwi.py) on the CPU: the order of the
checkpoints, segment recomputations, dense Krylov states, adjoint steps and seismogram
injections, checked end to end on a stand-in model whose step is a small linear map with a
known transpose.  The driver's gradient must equal the gradient torch's autograd takes
through the same forward loop, for every checkpoint budget, with and without dense states,
and for leap-frog's two levels (state and history vector in every checkpoint).
The stand-in only mirrors the call interface of ``Model``; the GPU arithmetic is covered by
tests/test_gpu_fwi.py."""
import types

import numpy as np
import pytest
import torch

from paper_2401_16322_gb300.fwi import FaberFWI

NV, NS, NREC = 12, 2, 3
REC = [1, 5, 9]


class StandIn:
    """U^{n+1} = U^n * (1 - dt m) + dt s_n per shot (m = c^2 elementwise on the single field),
    recording U^{n+1} at the receivers after each step; the adjoint of step n maps lambda to
    lambda * (1 - dt m) and adds lambda * (-dt U^{n-1}) to the gradient."""

    def __init__(self):
        self.torch = torch
        self.vector_elems = NV
        self.nshots = NS
        self.dtype = torch.float64
        self.device = "cpu"
        self.layout = types.SimpleNamespace(field_elems=NV, pitch=NV)
        self.nx, self.ny = NV, 1
        self.max_receivers = NREC
        self.capacity = 0
        self.seismo = None
        self.state = torch.zeros(NS * NV, dtype=torch.float64)
        self.work = torch.zeros(NS * 4 * NV, dtype=torch.float64)
        self.m = torch.zeros(NV, dtype=torch.float64)
        self.cursor = 0
        self.calls = []

    # set-up -------------------------------------------------------------------------
    def set_velocity(self, c):
        self.m = torch.tensor(np.asarray(c, dtype=np.float64).ravel() ** 2)

    def bind_seismogram(self, capacity):
        self.seismo = torch.zeros(NS * capacity * NREC, dtype=torch.float64)
        self.capacity = capacity

    def reset_state(self):
        self.state.zero_()
        self.cursor = 0

    def ensure_workspace(self, method, m=0):
        pass

    def sync(self):
        pass

    # forward --------------------------------------------------------------------------
    @staticmethod
    def source(t, s):
        return torch.tensor([np.sin(40.0 * t + s + q) for q in range(NV)], dtype=torch.float64)

    def _advance(self, t, dt):
        U = self.state.view(NS, NV)
        for s in range(NS):
            U[s] = U[s] * (1.0 - dt * self.m) + dt * self.source(t, s)
        if self.cursor < self.capacity:
            rec = self.seismo.view(NS, self.capacity, NREC)
            for s in range(NS):
                rec[s, self.cursor] = U[s, REC]
        self.cursor += 1

    def step(self, method, t, dt, degree, nsteps):
        assert nsteps == 1
        self.calls.append(("step", round(t / dt)))
        self._advance(t, dt)

    def step_krylov_dense(self, t, dt, m, dense):
        self.calls.append(("dense", round(t / dt)))
        flat = dense.view(-1)
        for q in range(4):                      # the stand-in's "dense states": U^{n-1}
            flat[q * NS * NV:(q + 1) * NS * NV].copy_(self.state)
        self._advance(t, dt)

    # adjoint --------------------------------------------------------------------------
    def _adjoint(self, dt, U_prev, lam, grad):
        L = lam.view(NS, NV)
        G = grad.view(NS, NV)
        P = U_prev.view(NS, NV)
        for s in range(NS):
            G[s] += L[s] * (-dt * P[s])
            L[s] = L[s] * (1.0 - dt * self.m)

    def adjoint_step(self, t, dt, degree, checkpoint, lam, grad, method="faber"):
        self.calls.append(("adj", round(t / dt)))
        self._adjoint(dt, checkpoint, lam, grad)

    def adjoint_step_krylov_dense(self, t, dt, m, dense, lam, grad):
        self.calls.append(("adj_dense", round(t / dt)))
        self._adjoint(dt, dense.reshape(-1)[:NS * NV], lam, grad)

    def adjoint_inject(self, lam, values):
        L = lam[:NS * NV].view(NS, NV)          # the first nshots vectors (level n)
        V = values.view(NS, NREC)
        for s in range(NS):
            L[s, REC] += V[s]

    def sum_shot_fields(self, per_shot, out):
        out.copy_(per_shot.view(NS, NV).sum(0))


def _autograd_gradient(c, d_obs, dt, nsteps):
    m = torch.tensor(np.asarray(c, dtype=np.float64).ravel() ** 2, requires_grad=True)
    U = [torch.zeros(NV, dtype=torch.float64) for _ in range(NS)]
    J = 0.0
    for n in range(nsteps):
        for s in range(NS):
            U[s] = U[s] * (1.0 - dt * m) + dt * StandIn.source(n * dt, s)
            J = J + 0.5 * ((U[s][REC] - d_obs[s, n]) ** 2).sum()
    J.backward()
    return m.grad.numpy()


@pytest.mark.parametrize("budget", [None, 1, 3, 4, 7])
@pytest.mark.parametrize("method,dense", [("faber", False), ("krylov", False), ("krylov", True)])
def test_driver_gradient_equals_autograd(budget, method, dense):
    dt, nsteps = 0.01, 9
    rng = np.random.default_rng(3)
    c = 2.0 + rng.random(NV)
    d_obs = torch.tensor(rng.standard_normal((NS, nsteps, NREC)), dtype=torch.float64)
    md = StandIn()
    fwi = FaberFWI(md, dt, 4, nsteps, NREC, budget=budget, method=method, dense_states=dense)
    seis = fwi.forward(c ** 2)
    grad = fwi.backward(seis - d_obs).numpy().ravel()
    want = _autograd_gradient(c, d_obs, dt, nsteps)
    assert np.allclose(grad, want, rtol=1e-12, atol=1e-14), np.abs(grad - want).max()
    # the adjoint ran once per step, from the last step back to the first
    adj = [n for k, n in md.calls if k in ("adj", "adj_dense")]
    assert adj == list(range(nsteps - 1, -1, -1))
    if dense:
        assert all(k != "adj" for k, _ in md.calls)
    if dense and budget is None:
        assert fwi.ckpt.shape[0] == 0                  # no checkpoint is read back
        assert [n for k, n in md.calls if k == "dense"] == list(range(nsteps))


class LeapfrogStandIn(StandIn):
    """Two-level stand-in: u^{n+1} = (2 - dt^2 m) u^n - u^{n-1} + dt^2 s_n, with u^{n-1} kept as
    the library keeps it (workspace vector 1 of each shot; u^{-1} = u^0 after a reset).  The
    adjoint takes the cotangents (a, b) of (u^n, u^{n-1}) in two vectors per shot to
    ((2 - dt^2 m) a + b, -a) and adds a (-dt^2 u^{n-1}) to the gradient."""

    def __init__(self):
        super().__init__()
        self.valid = False

    def reset_state(self):
        super().reset_state()
        self.valid = False

    def _history(self):
        return self.work.view(NS, self.work.numel() // (NS * NV), NV)[:, 0, :]

    def step(self, method, t, dt, degree, nsteps):
        assert method == "leapfrog" and nsteps == 1
        self.calls.append(("step", round(t / dt)))
        U = self.state.view(NS, NV)
        H = self._history()
        prev = H.clone() if self.valid else U.clone()
        H.copy_(U)
        for s in range(NS):
            U[s] = (2.0 - dt * dt * self.m) * U[s] - prev[s] + dt * dt * self.source(t, s)
        self.valid = True
        if self.cursor < self.capacity:
            rec = self.seismo.view(NS, self.capacity, NREC)
            for s in range(NS):
                rec[s, self.cursor] = U[s, REC]
        self.cursor += 1

    def adjoint_step(self, t, dt, degree, checkpoint, lam, grad, method="faber"):
        assert method == "leapfrog"
        self.calls.append(("adj", round(t / dt)))
        A = lam[:NS * NV].view(NS, NV)
        B = lam[NS * NV:2 * NS * NV].view(NS, NV)
        G = grad.view(NS, NV)
        P = checkpoint.view(NS, NV)
        for s in range(NS):
            G[s] += A[s] * (-dt * dt * P[s])
            a_new = (2.0 - dt * dt * self.m) * A[s] + B[s]
            B[s] = -A[s]
            A[s] = a_new


def _autograd_gradient_leapfrog(c, d_obs, dt, nsteps):
    m = torch.tensor(np.asarray(c, dtype=np.float64).ravel() ** 2, requires_grad=True)
    U = [torch.zeros(NV, dtype=torch.float64) for _ in range(NS)]
    Up = [u.clone() for u in U]
    J = 0.0
    for n in range(nsteps):
        for s in range(NS):
            nxt = (2.0 - dt * dt * m) * U[s] - Up[s] + dt * dt * StandIn.source(n * dt, s)
            Up[s], U[s] = U[s], nxt
            J = J + 0.5 * ((U[s][REC] - d_obs[s, n]) ** 2).sum()
    J.backward()
    return m.grad.numpy()


@pytest.mark.parametrize("budget", [None, 1, 2, 4, 7])
def test_leapfrog_driver_gradient_equals_autograd(budget):
    """Leap-frog carries two levels: checkpoints store the state and the history vector, and
    a segment's recomputation restores both."""
    dt, nsteps = 0.01, 11
    rng = np.random.default_rng(5)
    c = 2.0 + rng.random(NV)
    d_obs = torch.tensor(rng.standard_normal((NS, nsteps, NREC)), dtype=torch.float64)
    md = LeapfrogStandIn()
    fwi = FaberFWI(md, dt, 1, nsteps, NREC, budget=budget, method="leapfrog")
    seis = fwi.forward(c ** 2)
    grad = fwi.backward(seis - d_obs).numpy().ravel()
    want = _autograd_gradient_leapfrog(c, d_obs, dt, nsteps)
    assert np.allclose(grad, want, rtol=1e-12, atol=1e-14), np.abs(grad - want).max()
    assert [n for k, n in md.calls if k == "adj"] == list(range(nsteps - 1, -1, -1))


def test_dense_states_need_krylov():
    with pytest.raises(ValueError):
        FaberFWI(StandIn(), 0.01, 4, 5, NREC, method="faber", dense_states=True)

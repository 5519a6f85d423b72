"""Full-waveform-inversion gradient through the library's discrete adjoint.

The forward map takes m = c^2 (squared velocity at the nodes, [ny, nx]) to every shot's
seismogram (Faber, HORK or Krylov steps, Sec. 3.2, or leap-frog steps, Sec. 3.1).  The backward pass runs the exact discrete adjoint of
those steps (``ewv_adjoint_step``), injecting the seismogram cotangent at the receivers
(``ewv_adjoint_inject``), and returns dL/dm.  Forward states are checkpointed every
``stride`` steps (``ewv_checkpoint_stride``): with stride 1 every state is stored, which is
the memory N_mem = T/dt that the paper's large exponential steps reduce (Secs. 3.3, 6);
with stride k the states inside a segment are recomputed from its checkpoint.

All arithmetic runs in the library's kernels; this module allocates device buffers (torch)
and sequences the calls.
"""
import numpy as np

from .ewave import Model, checkpoint_stride


class FaberFWI:
    """Forward simulation with checkpoints and the adjoint gradient for one model
    (``method`` "faber": degree m; "hork": m stages; "krylov": dimension m, the adjoint the
    model's Krylov adjoint mode selects; "leapfrog": the two-step scheme with averaged
    damping, m ignored).

    Leap-frog carries two time levels: a checkpoint stores the state (level n) and the
    library's history vector (level n-1, workspace vector 1 of each shot), and the adjoint
    state has two vectors per shot (``ewv_adjoint_step``).

    ``dense_states`` (Krylov only): the adjoint of each step's exponential runs from the four
    dense states the forward step writes (``ewv_step_krylov_dense``) instead of recomputing
    the forward Arnoldi from a checkpoint.  With every step stored (no budget) the forward
    pass keeps them, 4 vectors per step in place of 1; with a budget a segment's dense states
    are recomputed from its checkpoint in the backward pass."""

    def __init__(self, model: Model, dt, degree, nsteps, nrec, budget=None, t0=0.0, method="faber",
                 dense_states=False):
        if method not in ("faber", "hork", "krylov", "leapfrog"):
            raise ValueError("the adjoint exists for the Faber, HORK, Krylov and leap-frog steps")
        if dense_states and method != "krylov":
            raise ValueError("dense states belong to the Krylov step")
        self.dense = bool(dense_states)
        self.method = method
        self.model = model
        self.dt, self.degree, self.nsteps, self.nrec, self.t0 = dt, degree, nsteps, nrec, t0
        self.stride = checkpoint_stride(nsteps, budget if budget else max(nsteps, 1))
        torch = model.torch
        nv = model.vector_elems
        self.levels = 2 if method == "leapfrog" else 1
        if method == "leapfrog":
            # one workspace for the forward steps and the adjoint: never rebound in between,
            # so the history vector survives
            model.ensure_workspace("adjoint_leapfrog", 0)
        self.nck = (nsteps + self.stride - 1) // self.stride
        ns = model.nshots
        # with dense states and every step stored, no checkpoint is read back
        nck = 0 if (self.dense and self.stride == 1) else self.nck
        self.ckpt = torch.zeros(nck, self.levels, ns * nv, dtype=model.dtype, device=model.device)
        self.seg = torch.zeros(0 if self.dense else self.stride, ns * nv, dtype=model.dtype,
                               device=model.device)
        # dense states [step, q, shot vectors]: every step's (no budget) or one segment's
        nxd = (nsteps if self.stride == 1 else self.stride) if self.dense else 0
        self.xd = torch.zeros(nxd, 4, ns * nv, dtype=model.dtype, device=model.device)

    def stored_bytes(self):
        """Device bytes of the stored forward states (checkpoints, segment and dense states)."""
        return sum(b.numel() * b.element_size() for b in (self.ckpt, self.seg, self.xd))

    def _history(self):
        """Leap-frog: the level n-1 vector of every shot (workspace vector 1), as a view."""
        md = self.model
        nv, ns = md.vector_elems, md.nshots
        per_shot = md.work.numel() // (ns * nv)
        return md.work.view(ns, per_shot, nv)[:, 0, :]

    def _save(self, k):
        md = self.model
        self.ckpt[k, 0].copy_(md.state)
        if self.levels == 2:
            nv, ns = md.vector_elems, md.nshots
            if k == 0:
                self.ckpt[k, 1].copy_(md.state)          # u^{-1} = u^0, w^{-1} = w^0
            else:
                self.ckpt[k, 1].view(ns, nv).copy_(self._history())

    def _restore(self, k):
        md = self.model
        md.state.copy_(self.ckpt[k, 0])
        if self.levels == 2:
            nv, ns = md.vector_elems, md.nshots
            self._history().copy_(self.ckpt[k, 1].view(ns, nv))

    def _set_m(self, m_c2):
        c = np.sqrt(np.asarray(m_c2.detach().double().cpu().numpy() if hasattr(m_c2, "detach") else m_c2,
                               dtype=np.float64))
        self.model.set_velocity(c)

    def forward(self, m_c2):
        """Seismograms [nshots, nsteps, nrec] (a copy) for squared velocity m_c2 [ny, nx]."""
        md = self.model
        self._set_m(m_c2)
        if md.capacity < self.nsteps:
            md.bind_seismogram(self.nsteps)
        md.reset_state()
        md.ensure_workspace(self.method, self.degree)
        for n in range(self.nsteps):
            if n % self.stride == 0 and self.ckpt.shape[0] > 0:
                self._save(n // self.stride)
            if self.dense and self.stride == 1:
                md.step_krylov_dense(self.t0 + n * self.dt, self.dt, self.degree, self.xd[n])
            else:
                md.step(self.method, self.t0 + n * self.dt, self.dt, self.degree, 1)
        md.sync()           # raises if the forward run produced a non-finite state
        s = md.seismo.view(md.nshots, md.capacity, md.max_receivers)[:, :self.nsteps, :self.nrec]
        return s.clone()

    def backward(self, grad_seis):
        """dL/dm [ny, nx] from the seismogram cotangent grad_seis [nshots, nsteps, nrec]."""
        md = self.model
        torch = md.torch
        nv, ns = md.vector_elems, md.nshots
        fe = md.layout.field_elems
        g = torch.zeros(ns, md.max_receivers * self.nsteps, dtype=md.dtype, device=md.device)
        g = g.view(ns, self.nsteps, md.max_receivers)
        g[:, :, :self.nrec] = grad_seis.to(md.dtype)
        lam = torch.zeros(self.levels * ns * nv, dtype=md.dtype, device=md.device)
        grad = torch.zeros(ns * fe, dtype=md.dtype, device=md.device)
        adj_ws = {"krylov": "adjoint_krylov", "leapfrog": "adjoint_leapfrog"}.get(self.method, "adjoint_faber")
        md.ensure_workspace(adj_ws, self.degree)
        md.adjoint_inject(lam, g[:, self.nsteps - 1, :].contiguous())
        for k in range(self.nck - 1, -1, -1):
            n0 = k * self.stride
            n1 = min(n0 + self.stride, self.nsteps)
            if self.dense and self.stride > 1:
                # recompute the segment's steps n0+1 .. n1 from its checkpoint, keeping the
                # dense states of each
                md.ensure_workspace(self.method, self.degree)
                self._restore(k)
                for n in range(n0, n1):
                    md.step_krylov_dense(self.t0 + n * self.dt, self.dt, self.degree, self.xd[n - n0])
                md.ensure_workspace(adj_ws, self.degree)
            if self.dense:
                for n in range(n1, n0, -1):      # adjoint of step n from its dense states
                    xd = self.xd[n - 1] if self.stride == 1 else self.xd[n - 1 - n0]
                    md.adjoint_step_krylov_dense(self.t0 + (n - 1) * self.dt, self.dt, self.degree, xd, lam, grad)
                    if n - 1 >= 1:
                        md.adjoint_inject(lam, g[:, n - 2, :].contiguous())
                continue
            # recompute the states U^{n0} .. U^{n1-1} of this segment from its checkpoint
            if self.stride > 1:
                md.ensure_workspace(self.method, self.degree)
                self._restore(k)
                for n in range(n0, n1):
                    self.seg[n - n0].copy_(md.state)
                    if n + 1 < n1:
                        md.step(self.method, self.t0 + n * self.dt, self.dt, self.degree, 1)
                md.ensure_workspace(adj_ws, self.degree)
            for n in range(n1, n0, -1):          # adjoint of step n: U^{n-1} -> U^n
                ck = self.seg[n - 1 - n0] if self.stride > 1 else self.ckpt[n - 1, 0]
                md.adjoint_step(self.t0 + (n - 1) * self.dt, self.dt, self.degree, ck, lam, grad,
                                self.method)
                if n - 1 >= 1:
                    md.adjoint_inject(lam, g[:, n - 2, :].contiguous())
        out = torch.zeros(fe, dtype=md.dtype, device=md.device)
        md.sum_shot_fields(grad, out)
        return out.view(md.ny, md.layout.pitch)[:, :md.nx]


def seismogram_fn():
    """torch.autograd.Function: m_c2 [ny, nx] -> seismograms, backward by the adjoint."""
    import torch

    class FaberSeismogram(torch.autograd.Function):
        @staticmethod
        def forward(ctx, m_c2, fwi):
            ctx.fwi = fwi
            ctx.device, ctx.dtype = m_c2.device, m_c2.dtype
            return fwi.forward(m_c2)

        @staticmethod
        def backward(ctx, grad_seis):
            g = ctx.fwi.backward(grad_seis)
            return g.to(device=ctx.device, dtype=ctx.dtype), None

    return FaberSeismogram

"""Thin Python binding of the ``libewave.so`` C ABI (include/ewave.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels.  PyTorch provides device memory (the caller-owned buffers of the ABI) and the CUDA
stream.  There is no CPU fallback: if the library is missing or no GPU is present, the
constructors raise.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libewave.so")

EWV_OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "BAD_SIZE_OR_ALIGNMENT", -3: "WORKSPACE_TOO_SMALL", -4: "CUDA_ERROR",
    -5: "NONFINITE", -6: "TIMEOUT", -7: "UNSUPPORTED", -8: "NOT_BOUND",
}
F32, F64 = 0, 1
METHOD = {"apply": 0, "faber": 1, "krylov": 2, "hork": 3, "rk32": 4, "rk44": 5, "leapfrog": 6,
          "adjoint_faber": 7, "adjoint_krylov": 8, "adjoint_leapfrog": 9, "krylov_adaptive": 10}
LEAPFROG_AVERAGED, LEAPFROG_LITERAL, LEAPFROG_DIFFERENCE = 0, 1, 2

# Every symbol include/ewave.h declares (checked by the tests).
EXPORTS = [
    "ewv_sync", "ewv_batch_sync", "ewv_debug_set_wait_limit", "ewv_set_krylov_adjoint",
    "ewv_step_krylov_adaptive", "ewv_batch_step_krylov_adaptive",
    "ewv_create_model", "ewv_destroy_model", "ewv_set_stream", "ewv_layout",
    "ewv_workspace_bytes", "ewv_bind_buffers", "ewv_bind_workspace", "ewv_bind_seismogram",
    "ewv_reset_recording", "ewv_set_velocity", "ewv_set_source_receivers",
    "ewv_set_faber_ellipse", "ewv_get_faber_ellipse", "ewv_set_state", "ewv_get_state",
    "ewv_pack_vector", "ewv_unpack_vector", "ewv_apply_operator", "ewv_step_faber",
    "ewv_step_krylov", "ewv_step_rk", "ewv_step_leapfrog", "ewv_set_leapfrog_variant",
    "ewv_create_batch", "ewv_destroy_batch", "ewv_batch_set_stream", "ewv_batch_step_faber",
    "ewv_batch_step_krylov", "ewv_batch_step_rk", "ewv_batch_step_leapfrog", "ewv_last_error",
    "ewv_batch_last_error", "ewv_version", "ewv_launch_count", "ewv_enable_kernel_timing",
    "ewv_kernel_timing", "ewv_batch_enable_kernel_timing", "ewv_batch_kernel_timing", "ewv_reset_state",
    "ewv_faber_step_noalloc", "ewv_adjoint_step", "ewv_adjoint_inject", "ewv_checkpoint_stride",
    "ewv_step_krylov_dense", "ewv_adjoint_step_krylov_dense", "ewv_debug_set_column_kernel",
    "ewv_sum_shot_fields", "ewv_enable_graphs", "ewv_batch_enable_graphs",
    "ewv_set_kernel_variant", "ewv_kernel_variant", "ewv_batch_set_kernel_variant",
    "ewv_batch_kernel_variant", "ewv_set_source_receivers3d", "ewv_set_storage_rounding",
    "ewv_set_krylov_window",
    "ewv_set_hork_form",
]


class EwaveError(RuntimeError):
    pass


class ModelDesc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("dx", ctypes.c_double), ("fd_order", ctypes.c_int), ("pml_width", ctypes.c_int),
                ("beta0", ctypes.c_double), ("free_surface", ctypes.c_int),
                ("precision", ctypes.c_int), ("nshots", ctypes.c_int),
                ("src_taylor_p", ctypes.c_int), ("max_receivers", ctypes.c_int),
                ("nz", ctypes.c_int)]


class NoallocFaberArgs(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("pitch", ctypes.c_int),
                ("dx", ctypes.c_double), ("fd_order", ctypes.c_int), ("pml_width", ctypes.c_int),
                ("beta0", ctypes.c_double), ("free_surface", ctypes.c_int),
                ("has_source", ctypes.c_int), ("src_i", ctypes.c_int), ("src_j", ctypes.c_int),
                ("src_taylor_p", ctypes.c_int), ("f_peak", ctypes.c_double), ("t0", ctypes.c_double),
                ("amp", ctypes.c_double), ("gamma", ctypes.c_double), ("c0", ctypes.c_double),
                ("c1", ctypes.c_double)]


NOALLOC_MAX_FIELD_ELEMS = 1 << 19


class LayoutInfo(ctypes.Structure):
    _fields_ = [("pitch", ctypes.c_int), ("elem_bytes", ctypes.c_int),
                ("field_elems", ctypes.c_size_t), ("vector_bytes", ctypes.c_size_t),
                ("state_bytes", ctypes.c_size_t), ("params_bytes", ctypes.c_size_t),
                ("compact_n", ctypes.c_size_t)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libewave.so (in-tree build).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise EwaveError(f"{path} is missing: build it with `python -m paper_2401_16322_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    dp = ctypes.POINTER(ctypes.c_double)
    ip32 = ctypes.POINTER(ctypes.c_int32)
    sig = {
        "ewv_create_model": ([ctypes.POINTER(ModelDesc), ctypes.POINTER(vp)], i),
        "ewv_destroy_model": ([vp], i),
        "ewv_set_stream": ([vp, vp], i),
        "ewv_layout": ([vp, ctypes.POINTER(LayoutInfo)], i),
        "ewv_workspace_bytes": ([vp, i, i, ctypes.POINTER(sz)], i),
        "ewv_bind_buffers": ([vp, vp, sz, vp, sz, vp, sz], i),
        "ewv_bind_workspace": ([vp, vp, sz], i),
        "ewv_bind_seismogram": ([vp, vp, sz, i], i),
        "ewv_reset_recording": ([vp], i),
        "ewv_set_velocity": ([vp, dp, sz], i),
        "ewv_set_source_receivers": ([vp, i, d, d, d, d, d, i, dp, ip32, ip32], i),
        "ewv_set_source_receivers3d": ([vp, i, d, d, d, d, d, d, i, dp, ip32, ip32], i),
        "ewv_set_storage_rounding": ([vp, i], i),
        "ewv_set_krylov_window": ([vp, i], i),
        "ewv_set_hork_form": ([vp, i], i),
        "ewv_set_faber_ellipse": ([vp, d, d, d], i),
        "ewv_get_faber_ellipse": ([vp, dp, dp, dp], i),
        "ewv_set_state": ([vp, i, dp, sz], i),
        "ewv_get_state": ([vp, i, dp, sz], i),
        "ewv_pack_vector": ([vp, dp, sz, vp], i),
        "ewv_unpack_vector": ([vp, vp, dp, sz], i),
        "ewv_apply_operator": ([vp, i, vp, vp], i),
        "ewv_step_faber": ([vp, d, d, i, i], i),
        "ewv_step_krylov": ([vp, d, d, i, i, ctypes.POINTER(i)], i),
        "ewv_step_rk": ([vp, d, d, i, i, i], i),
        "ewv_step_leapfrog": ([vp, d, d, i], i),
        "ewv_set_leapfrog_variant": ([vp, i], i),
        "ewv_create_batch": ([ctypes.POINTER(vp), i, ctypes.POINTER(vp)], i),
        "ewv_destroy_batch": ([vp], i),
        "ewv_batch_set_stream": ([vp, vp], i),
        "ewv_batch_step_faber": ([vp, d, d, i, i], i),
        "ewv_batch_step_krylov": ([vp, d, d, i, i, ctypes.POINTER(i)], i),
        "ewv_batch_step_rk": ([vp, d, d, i, i, i], i),
        "ewv_batch_step_leapfrog": ([vp, d, d, i], i),
        "ewv_last_error": ([vp], ctypes.c_char_p),
        "ewv_batch_last_error": ([vp], ctypes.c_char_p),
        "ewv_version": ([], ctypes.c_char_p),
        "ewv_launch_count": ([vp, ctypes.POINTER(ctypes.c_longlong)], i),
        "ewv_reset_state": ([vp], i),
        "ewv_adjoint_step": ([vp, i, d, d, i, vp, vp, vp], i),
        "ewv_step_krylov_dense": ([vp, d, d, i, vp], i),
        "ewv_adjoint_step_krylov_dense": ([vp, d, d, i, vp, vp, vp], i),
        "ewv_adjoint_inject": ([vp, vp, vp], i),
        "ewv_checkpoint_stride": ([i, i, ctypes.POINTER(i)], i),
        "ewv_sum_shot_fields": ([vp, vp, vp], i),
        "ewv_enable_graphs": ([vp, i], i),
        "ewv_set_kernel_variant": ([vp, i], i),
        "ewv_kernel_variant": ([vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                ctypes.POINTER(i), dp], i),
        "ewv_batch_set_kernel_variant": ([vp, i], i),
        "ewv_batch_kernel_variant": ([vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                      ctypes.POINTER(i), dp], i),
        "ewv_batch_enable_graphs": ([vp, i], i),
        "ewv_faber_step_noalloc": ([ctypes.POINTER(NoallocFaberArgs), vp, vp, d, d, i, i, vp], i),
        "ewv_enable_kernel_timing": ([vp, i], i),
        "ewv_kernel_timing": ([vp, dp, ctypes.POINTER(ctypes.c_longlong)], i),
        "ewv_batch_enable_kernel_timing": ([vp, i], i),
        "ewv_batch_kernel_timing": ([vp, dp, ctypes.POINTER(ctypes.c_longlong)], i),
        "ewv_sync": ([vp], i),
        "ewv_batch_sync": ([vp], i),
        "ewv_debug_set_wait_limit": ([ctypes.c_ulonglong], i),
        "ewv_debug_set_column_kernel": ([i], i),
        "ewv_set_krylov_adjoint": ([vp, i], i),
        "ewv_step_krylov_adaptive": ([vp, d, d, d, i, i, i, ctypes.POINTER(i)], i),
        "ewv_batch_step_krylov_adaptive": ([vp, d, d, d, i, i, i, ctypes.POINTER(i)], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


# persistent-pass variants the autotuner times (EWV_NUM_KERNEL_VARIANTS)
NUM_KERNEL_VARIANTS = 15


def _variant(fn, h, check):
    v, by, nw, nst = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    us = (ctypes.c_double * NUM_KERNEL_VARIANTS)()
    check(fn(h, ctypes.byref(v), ctypes.byref(by), ctypes.byref(nw), ctypes.byref(nst), us))
    return {"variant": v.value, "tile": [64, by.value], "consumer_warps": nw.value,
            "stages": nst.value, "probe_us": list(us)}


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Model:
    """One velocity model with ``nshots`` shots, its device buffers held as torch tensors.
    With ``nz`` it is three-dimensional (grid nz x ny x nx, six fields: psi added)."""

    def __init__(self, nx, ny, dx, order=8, pml=40, beta0=0.0, free_surface=True,
                 precision="f32", nshots=1, p=12, max_receivers=0, device=None, stream=None,
                 nz=None):
        import torch
        if not torch.cuda.is_available():
            raise EwaveError("a CUDA device is required (the library has no CPU path)")
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device(device or "cuda")
        self.prec = F64 if precision in ("f64", "float64", F64) else F32
        self.dtype = torch.float64 if self.prec == F64 else torch.float32
        self.nx, self.ny, self.dx, self.nshots = nx, ny, dx, nshots
        self.nz = nz
        self.dims = 3 if nz else 2
        self.max_receivers = max_receivers
        d = ModelDesc(self.dims, nx, ny, dx, order, pml, beta0, int(bool(free_surface)), self.prec,
                      nshots, p, max_receivers, nz or 1)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            self._check(self.lib.ewv_create_model(ctypes.byref(d), ctypes.byref(h)), "create_model")
        self.h = h
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._check(self.lib.ewv_set_stream(self.h, ctypes.c_void_p(self.stream.cuda_stream)))
        lay = LayoutInfo()
        self._check(self.lib.ewv_layout(self.h, ctypes.byref(lay)))
        self.layout = lay
        self.n = lay.compact_n
        ne = lay.elem_bytes
        self.state = torch.zeros(lay.state_bytes // ne, dtype=self.dtype, device=self.device)
        self.params = torch.zeros(lay.params_bytes // ne, dtype=self.dtype, device=self.device)
        self.work = None
        self.seismo = None
        self.capacity = 0
        self._check(self.lib.ewv_bind_buffers(self.h, ctypes.c_void_p(self.state.data_ptr()),
                                              lay.state_bytes, ctypes.c_void_p(self.params.data_ptr()),
                                              lay.params_bytes, None, 0))

    # ---------------------------------------------------------------- helpers
    def _check(self, rc, what=""):
        if rc != EWV_OK:
            msg = ""
            if getattr(self, "h", None) is not None and self.h.value:
                msg = self.lib.ewv_last_error(self.h).decode()
            raise EwaveError(f"{what or 'ewave'}: {ERRORS.get(rc, rc)} {msg}")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.ewv_destroy_model(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def vector_elems(self):
        return self.layout.vector_bytes // self.layout.elem_bytes

    def new_vector(self):
        return self.torch.zeros(self.vector_elems, dtype=self.dtype, device=self.device)

    # ---------------------------------------------------------------- inputs
    def set_velocity(self, c):
        c = np.ascontiguousarray(c, dtype=np.float64)
        self._check(self.lib.ewv_set_velocity(self.h, _dptr(c), c.size), "set_velocity")

    def set_source_receivers(self, shot, sx, sy, f_peak, t0, amp=1.0, rec=None):
        rec = np.zeros((0, 2)) if rec is None else np.ascontiguousarray(rec, dtype=np.float64)
        nrec = rec.shape[0]
        si = np.zeros(2, dtype=np.int32)
        ri = np.zeros(max(2 * nrec, 1), dtype=np.int32)
        self._check(self.lib.ewv_set_source_receivers(
            self.h, shot, sx, sy, f_peak, t0, amp, nrec, _dptr(rec) if nrec else None,
            si.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            ri.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "set_source_receivers")
        return si, ri[:2 * nrec].reshape(nrec, 2)

    def set_source_receivers3d(self, shot, sx, sy, sz, f_peak, t0, amp=1.0, rec=None):
        """3D model: source at (sx, sy, depth sz), receivers as (x, y, depth) rows."""
        rec = np.zeros((0, 3)) if rec is None else np.ascontiguousarray(rec, dtype=np.float64)
        nrec = rec.shape[0]
        si = np.zeros(3, dtype=np.int32)
        ri = np.zeros(max(3 * nrec, 1), dtype=np.int32)
        self._check(self.lib.ewv_set_source_receivers3d(
            self.h, shot, sx, sy, sz, f_peak, t0, amp, nrec, _dptr(rec) if nrec else None,
            si.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            ri.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "set_source_receivers3d")
        return si, ri[:3 * nrec].reshape(nrec, 3)

    def set_hork_form(self, form):
        """'low-storage' (default, the paper's stages) or 'horner' evaluation of the HORK
        polynomial (fewer bytes per pass, less accurate in FP32 at large steps)."""
        code = {"horner": 0, "low-storage": 1}[form]
        self._check(self.lib.ewv_set_hork_form(self.h, code), "hork_form")

    def set_krylov_adjoint(self, mode):
        """'exact' (default): reverse mode through the computed Krylov step; 'exponential':
        the adjoint of exp(dt H~), which the step approximates."""
        self._check(self.lib.ewv_set_krylov_adjoint(self.h, {"exact": 0, "exponential": 1}[mode]),
                    "krylov_adjoint")

    def set_krylov_window(self, q):
        """Orthogonalise each Krylov vector against the q most recent ones only (0: all)."""
        self._check(self.lib.ewv_set_krylov_window(self.h, int(q)), "krylov_window")

    def set_storage_rounding(self, bf16):
        """Round every stored integrator vector to bfloat16 (storage-precision experiment)."""
        self._check(self.lib.ewv_set_storage_rounding(self.h, 1 if bf16 else 0), "storage_rounding")

    def set_faber_ellipse(self, gamma, c0, c1):
        self._check(self.lib.ewv_set_faber_ellipse(self.h, gamma, c0, c1))

    def faber_ellipse(self):
        g, c0, c1 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.ewv_get_faber_ellipse(self.h, ctypes.byref(g), ctypes.byref(c0),
                                                   ctypes.byref(c1)))
        return g.value, c0.value, c1.value

    def ensure_workspace(self, method, m=0):
        need = ctypes.c_size_t()
        self._check(self.lib.ewv_workspace_bytes(self.h, METHOD[method], m, ctypes.byref(need)))
        have = 0 if self.work is None else self.work.numel() * self.layout.elem_bytes
        if need.value > have:
            self.work = self.torch.zeros(need.value // self.layout.elem_bytes, dtype=self.dtype,
                                         device=self.device)
            self._check(self.lib.ewv_bind_workspace(self.h, ctypes.c_void_p(self.work.data_ptr()),
                                                    need.value))

    def bind_seismogram(self, capacity):
        n = max(self.nshots * capacity * self.max_receivers, 1)
        self.seismo = self.torch.zeros(n, dtype=self.dtype, device=self.device)
        self.capacity = capacity
        self._check(self.lib.ewv_bind_seismogram(self.h, ctypes.c_void_p(self.seismo.data_ptr()),
                                                 n * self.layout.elem_bytes, capacity))

    def reset_state(self):
        self._check(self.lib.ewv_reset_state(self.h), "reset_state")

    def reset_recording(self):
        self._check(self.lib.ewv_reset_recording(self.h))

    def seismogram(self, shot, nrec, nsamples):
        self.stream.synchronize()
        s = self.seismo.view(self.nshots, self.capacity, self.max_receivers)
        return s[shot, :nsamples, :nrec].double().cpu().numpy()

    # ---------------------------------------------------------------- state
    def set_state(self, shot, compact):
        x = np.ascontiguousarray(compact, dtype=np.float64)
        self._check(self.lib.ewv_set_state(self.h, shot, _dptr(x), x.size), "set_state")

    def get_state(self, shot):
        out = np.zeros(self.n)
        self._check(self.lib.ewv_get_state(self.h, shot, _dptr(out), out.size), "get_state")
        return out

    def pack(self, compact, dev):
        x = np.ascontiguousarray(compact, dtype=np.float64)
        self._check(self.lib.ewv_pack_vector(self.h, _dptr(x), x.size, ctypes.c_void_p(dev.data_ptr())))

    def unpack(self, dev):
        out = np.zeros(self.n)
        self._check(self.lib.ewv_unpack_vector(self.h, ctypes.c_void_p(dev.data_ptr()), _dptr(out),
                                               out.size))
        return out

    # ---------------------------------------------------------------- compute
    def apply_device(self, x, y, transpose=False):
        self._check(self.lib.ewv_apply_operator(self.h, int(transpose), ctypes.c_void_p(x.data_ptr()),
                                                ctypes.c_void_p(y.data_ptr())), "apply_operator")

    def apply(self, compact, transpose=False):
        x, y = self.new_vector(), self.new_vector()
        self.pack(compact, x)
        self.apply_device(x, y, transpose)
        return self.unpack(y)

    def step_faber(self, t, dt, degree, nsteps=1):
        self.ensure_workspace("faber", degree)
        self._check(self.lib.ewv_step_faber(self.h, t, dt, degree, nsteps), "step_faber")

    def step_krylov(self, t, dt, m, nsteps=1):
        self.ensure_workspace("krylov", m)
        info = ctypes.c_int(0)
        self._check(self.lib.ewv_step_krylov(self.h, t, dt, m, nsteps, ctypes.byref(info)), "step_krylov")
        return info.value

    def step_krylov_dense(self, t, dt, m, dense):
        """One Krylov step that also writes its four dense states x(tau_q dt) (4-point
        Gauss-Legendre nodes tau_q on [0, 1]) into ``dense``: 4 nshots padded vectors, [q][shot]
        (the input of adjoint_step_krylov_dense)."""
        self._need("dense", dense, 4 * self.nshots * self.vector_elems)
        self.ensure_workspace("krylov", m)
        self._check(self.lib.ewv_step_krylov_dense(self.h, t, dt, m, ctypes.c_void_p(dense.data_ptr())),
                    "step_krylov_dense")

    def step_krylov_adaptive(self, t, dt, tol, m_min=1, m_max=30, nsteps=1):
        """Adaptive Krylov steps (dimension and substeps chosen per shot to meet ``tol``);
        returns {"substeps", "matvecs", "max_dim"} summed over shots and steps."""
        self.ensure_workspace("krylov_adaptive", m_max)
        st = (ctypes.c_int * 3)()
        self._check(self.lib.ewv_step_krylov_adaptive(self.h, t, dt, tol, m_min, m_max, nsteps, st),
                    "step_krylov_adaptive")
        return {"substeps": st[0], "matvecs": st[1], "max_dim": st[2]}

    def step_rk(self, t, dt, scheme, stages=0, nsteps=1):
        self.ensure_workspace(scheme, stages)
        self._check(self.lib.ewv_step_rk(self.h, t, dt, METHOD[scheme], stages, nsteps), "step_rk")

    def set_leapfrog_variant(self, variant):
        """LEAPFROG_AVERAGED (default), LEAPFROG_LITERAL or LEAPFROG_DIFFERENCE (2D)."""
        self._check(self.lib.ewv_set_leapfrog_variant(self.h, int(variant)), "leapfrog_variant")

    def step_leapfrog(self, t, dt, nsteps=1, variant=None):
        """Leap-frog steps; ``variant`` (if given) is set first, else the model's is kept."""
        self.ensure_workspace("leapfrog")
        if variant is not None:
            self.set_leapfrog_variant(variant)
        self._check(self.lib.ewv_step_leapfrog(self.h, t, dt, nsteps), "step_leapfrog")

    def step(self, method, t, dt, m=0, nsteps=1):
        if method == "faber":
            return self.step_faber(t, dt, m, nsteps)
        if method == "krylov":
            return self.step_krylov(t, dt, m, nsteps)
        if method in ("hork", "rk32", "rk44"):
            return self.step_rk(t, dt, method, m, nsteps)
        if method == "leapfrog":
            return self.step_leapfrog(t, dt, nsteps)
        raise ValueError(method)

    def launch_count(self):
        c = ctypes.c_longlong()
        self._check(self.lib.ewv_launch_count(self.h, ctypes.byref(c)))
        return c.value

    def sync(self):
        """Wait for the model's GPU work; raise on a non-finite state or a timed-out wait."""
        self._check(self.lib.ewv_sync(self.h), "sync")

    # ---------------------------------------------------------------- adjoint
    def adjoint_step(self, t, dt, degree, checkpoint, adj, grad, method="faber"):
        """lambda <- (dPhi/dU)^T lambda, grad += (dPhi/dm)^T lambda for one Faber / HORK /
        Krylov / leap-frog step (Krylov: the exact discrete adjoint, or the adjoint of the
        step's exponential after set_krylov_adjoint('exponential')).  Leap-frog: ``adj``
        holds 2 nshots vectors (cotangents of level n, then of w at level n-1)."""
        ns, nv, fe = self.nshots, self.vector_elems, self.layout.field_elems
        levels = 2 if method == "leapfrog" else 1
        for name, buf, need in (("checkpoint", checkpoint, ns * nv), ("adj", adj, levels * ns * nv),
                                ("grad", grad, ns * fe)):
            self._need(name, buf, need)
        self.ensure_workspace({"krylov": "adjoint_krylov", "leapfrog": "adjoint_leapfrog"}.get(
            method, "adjoint_faber"), degree)
        self._check(self.lib.ewv_adjoint_step(self.h, METHOD[method], t, dt, degree,
                                              ctypes.c_void_p(checkpoint.data_ptr()),
                                              ctypes.c_void_p(adj.data_ptr()),
                                              ctypes.c_void_p(grad.data_ptr())), "adjoint_step")

    def adjoint_step_krylov_dense(self, t, dt, m, dense, adj, grad):
        """The adjoint of one Krylov step's exponential from the forward step's dense states
        (step_krylov_dense) instead of a checkpoint: no forward Arnoldi is recomputed."""
        ns, nv, fe = self.nshots, self.vector_elems, self.layout.field_elems
        for name, buf, need in (("dense", dense, 4 * ns * nv), ("adj", adj, ns * nv), ("grad", grad, ns * fe)):
            self._need(name, buf, need)
        self.ensure_workspace("adjoint_krylov", m)
        self._check(self.lib.ewv_adjoint_step_krylov_dense(self.h, t, dt, m, ctypes.c_void_p(dense.data_ptr()),
                                                           ctypes.c_void_p(adj.data_ptr()),
                                                           ctypes.c_void_p(grad.data_ptr())),
                    "adjoint_step_krylov_dense")

    def _need(self, name, buf, need):
        if buf.numel() < need or buf.dtype != self.dtype or not buf.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor of at least {need} {self.dtype} elements "
                             f"(got {buf.numel()} {buf.dtype} on {buf.device})")

    def adjoint_inject(self, adj, values):
        self._check(self.lib.ewv_adjoint_inject(self.h, ctypes.c_void_p(adj.data_ptr()),
                                                ctypes.c_void_p(values.data_ptr())), "adjoint_inject")

    def sum_shot_fields(self, per_shot, out):
        self._check(self.lib.ewv_sum_shot_fields(self.h, ctypes.c_void_p(per_shot.data_ptr()),
                                                 ctypes.c_void_p(out.data_ptr())), "sum_shot_fields")

    def enable_graphs(self, on=True):
        self._check(self.lib.ewv_enable_graphs(self.h, int(on)))

    def set_kernel_variant(self, v):
        self._check(self.lib.ewv_set_kernel_variant(self.h, v))

    def kernel_variant(self):
        return _variant(self.lib.ewv_kernel_variant, self.h, self._check)

    def enable_kernel_timing(self, on=True):
        self._check(self.lib.ewv_enable_kernel_timing(self.h, int(on)))

    def kernel_timing(self):
        """(total ms, launches) of the stencil passes since the last read."""
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        self._check(self.lib.ewv_kernel_timing(self.h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value


def checkpoint_stride(nsteps, budget):
    """Checkpoint every stride-th step so that at most ``budget`` states are stored."""
    out = ctypes.c_int()
    rc = load_library().ewv_checkpoint_stride(nsteps, budget, ctypes.byref(out))
    if rc != EWV_OK:
        raise EwaveError(f"checkpoint_stride: {ERRORS.get(rc, rc)}")
    return out.value


def debug_set_wait_limit(ns):
    """Testing aid: wait limit (ns, default 1e9) of the 2D FP32 TMA pass's pipeline waits and
    of the Gram-Schmidt column kernel's grid barriers."""
    rc = load_library().ewv_debug_set_wait_limit(int(ns))
    if rc != EWV_OK:
        raise EwaveError(f"debug_set_wait_limit: {ERRORS.get(rc, rc)}")


def debug_set_column_kernel(enable):
    """Testing aid: run the Krylov Gram-Schmidt steps on the column kernel (True, default,
    where the engine's chunks fit one co-resident grid) or on the flat passes (False)."""
    rc = load_library().ewv_debug_set_column_kernel(1 if enable else 0)
    if rc != EWV_OK:
        raise EwaveError(f"debug_set_column_kernel: {ERRORS.get(rc, rc)}")


def faber_step_noalloc(args, state, c2, t, dt, degree, nsteps=1, stream=None):
    """Allocation-free Faber step (``ewv_faber_step_noalloc``) on caller-owned FP32 device
    tensors ``state`` (padded state vector) and ``c2``; returns the status code.

    For callers that cannot allocate device memory: the library keeps the work vectors in
    a fixed device array (grids up to ny * pitch = NOALLOC_MAX_FIELD_ELEMS)."""
    import torch
    lib = load_library()
    s = stream if stream is not None else torch.cuda.current_stream()
    return lib.ewv_faber_step_noalloc(ctypes.byref(args), ctypes.c_void_p(state.data_ptr()),
                                      ctypes.c_void_p(c2.data_ptr()), t, dt, degree, nsteps,
                                      ctypes.c_void_p(s.cuda_stream))


class Batch:
    """Several models (uneven sizes allowed) stepped in the same kernel launches."""

    def __init__(self, models, stream=None):
        self.lib = load_library()
        self.models = list(models)
        arr = (ctypes.c_void_p * len(self.models))(*[m.h.value for m in self.models])
        h = ctypes.c_void_p()
        rc = self.lib.ewv_create_batch(arr, len(self.models), ctypes.byref(h))
        if rc != EWV_OK:
            raise EwaveError(f"create_batch: {ERRORS.get(rc, rc)}")
        self.h = h
        if stream is not None:
            self.lib.ewv_batch_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream))

    def _check(self, rc, what):
        if rc != EWV_OK:
            raise EwaveError(f"{what}: {ERRORS.get(rc, rc)} {self.lib.ewv_batch_last_error(self.h).decode()}")

    def step(self, method, t, dt, m=0, nsteps=1):
        for md in self.models:
            md.ensure_workspace(method, m)
        if method == "faber":
            self._check(self.lib.ewv_batch_step_faber(self.h, t, dt, m, nsteps), "batch_step_faber")
        elif method == "krylov":
            info = ctypes.c_int(0)
            self._check(self.lib.ewv_batch_step_krylov(self.h, t, dt, m, nsteps, ctypes.byref(info)),
                        "batch_step_krylov")
            return info.value
        elif method in ("hork", "rk32", "rk44"):
            self._check(self.lib.ewv_batch_step_rk(self.h, t, dt, METHOD[method], m, nsteps), "batch_step_rk")
        elif method == "leapfrog":
            self._check(self.lib.ewv_batch_step_leapfrog(self.h, t, dt, nsteps), "batch_step_leapfrog")
        else:
            raise ValueError(method)

    def step_krylov_adaptive(self, t, dt, tol, m_min=1, m_max=30, nsteps=1):
        for md in self.models:
            md.ensure_workspace("krylov_adaptive", m_max)
        st = (ctypes.c_int * 3)()
        self._check(self.lib.ewv_batch_step_krylov_adaptive(self.h, t, dt, tol, m_min, m_max, nsteps, st),
                    "batch_step_krylov_adaptive")
        return {"substeps": st[0], "matvecs": st[1], "max_dim": st[2]}

    def enable_graphs(self, on=True):
        self._check(self.lib.ewv_batch_enable_graphs(self.h, int(on)), "graphs")

    def set_kernel_variant(self, v):
        self._check(self.lib.ewv_batch_set_kernel_variant(self.h, v), "variant")

    def kernel_variant(self):
        return _variant(self.lib.ewv_batch_kernel_variant, self.h, lambda rc, w="": self._check(rc, "variant"))

    def enable_kernel_timing(self, on=True):
        self._check(self.lib.ewv_batch_enable_kernel_timing(self.h, int(on)), "timing")

    def kernel_timing(self):
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        self._check(self.lib.ewv_batch_kernel_timing(self.h, ctypes.byref(ms), ctypes.byref(n)), "timing")
        return ms.value, n.value

    def launch_count(self):
        return sum(m.launch_count() for m in self.models[:1])

    def sync(self):
        """Wait for the batch's GPU work; raise on a non-finite state or a timed-out wait."""
        self._check(self.lib.ewv_batch_sync(self.h), "batch_sync")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.ewv_destroy_batch(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

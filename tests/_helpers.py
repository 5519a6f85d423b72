"""Shared test helpers: build the oracle model and the GPU model from the same seeded
inputs, and compare with the tolerances of the acceptance criteria."""
import numpy as np

from oracle.faber import ellipse_params
from oracle.model import Model as OModel
from oracle.model import default_beta0, flatten, unflatten
from oracle.simulate import rel_l2

# Acceptance tolerances (relative L2): FP64 path vs the FP64 oracle; FP32 path per step.
TOL = {"f64": 1e-12, "f32": 1e-5}
TOL_SEISMO_F32 = 1e-4


def oracle_model(nx, ny, c, order=8, pml=10, fs=True, dx=10.0, beta0=None):
    b0 = default_beta0(float(np.max(c)), pml, dx) if beta0 is None else beta0
    return OModel(nx, ny, dx, order, pml, b0, fs, c)


def gpu_model(om, precision="f64", nshots=1, p=12, max_receivers=0):
    from paper_2401_16322_gb300 import Model
    g = Model(om.nx, om.ny, om.dx, om.order, om.pml, om.beta0, om.free_surface,
              precision=precision, nshots=nshots, p=p, max_receivers=max_receivers)
    g.set_velocity(om.c)
    return g


def rel_l2_fields(got, ref, shapes, floor=1e-3):
    """Relative L2 error of every field of two flattened states (fields in ``shapes`` order):
    |got_f - ref_f| / max(|ref_f|, floor |ref|), so that an error in a field with a small norm
    does not hide behind the others."""
    out, o = [], 0
    total = float(np.linalg.norm(ref))
    for sh in shapes:
        n = int(np.prod(sh))
        g, r = got[o:o + n], ref[o:o + n]
        out.append(float(np.linalg.norm(g - r) / max(np.linalg.norm(r), floor * total)))
        o += n
    return out


def oracle_ellipse(om):
    return ellipse_params(om.c_max, om.beta0, om.dx, om.order, free_surface=om.free_surface)


__all__ = ["TOL", "TOL_SEISMO_F32", "oracle_model", "gpu_model", "oracle_ellipse", "flatten",
           "unflatten", "rel_l2", "rel_l2_fields"]

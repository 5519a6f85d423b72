"""GPU parity of the three-dimensional path (the auxiliary-field PML form of Eq. 1 used for the
400^3 workload, oracle/wave3d_pml.py) against the oracle, through the C ABI: H x on ragged grids
(FP64 1e-12, FP32 1e-5, whole state and every field on its own), every integrator with the
source active and receivers recorded, and bit-exact node indices."""
import numpy as np
import pytest

from _helpers import TOL, flatten, rel_l2, rel_l2_fields
from oracle import faber, krylov, rk
from oracle import wave3d as W
from oracle import wave3d_pml as PML
from oracle.model import default_beta0, unflatten
from paper_2401_16322_gb300.workloads import layered3d, smooth_random_state

pytestmark = pytest.mark.gpu


def _models(nx, ny, nz, prec, fs=True, order=8, pml=6, p=10, max_receivers=0, seed=3):
    from paper_2401_16322_gb300 import Model
    c = layered3d(nx, ny, nz, seed)
    b0 = default_beta0(float(c.max()), pml, 10.0)
    om = PML.Model3DPML(nx, ny, nz, 10.0, order, pml, b0, fs, c)
    g = Model(nx, ny, 10.0, order, pml, b0, fs, precision=prec, p=p, max_receivers=max_receivers,
              nz=nz)
    g.set_velocity(c)
    return om, g


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("shape,fs,order", [((70, 37, 45), True, 8), ((67, 19, 34), False, 8),
                                            ((40, 21, 35), False, 4)])
def test_operator_matches_oracle(prec, shape, fs, order):
    nx, ny, nz = shape          # ragged in every tile direction (64 x 16 x 32 tiles)
    om, g = _models(nx, ny, nz, prec, fs=fs, order=order)
    x = flatten(smooth_random_state(om.field_shapes(), 17))
    ref = flatten(PML.apply_H3p(om, unflatten(om, x)))
    got = g.apply(x)
    assert rel_l2(got, ref) < TOL[prec]
    assert max(rel_l2_fields(got, ref, om.field_shapes())) < TOL[prec], rel_l2_fields(got, ref, om.field_shapes())
    g.close()


def test_transpose_and_adjoint_are_rejected_in_3d():
    from paper_2401_16322_gb300.ewave import EwaveError
    om, g = _models(20, 17, 18, "f64")
    with pytest.raises(EwaveError, match="UNSUPPORTED"):
        g.apply(np.zeros(om.n), transpose=True)
    g.close()


NX, NY, NZ = 44, 23, 38


def _setup(prec, p=10):
    rec = np.array([[x * 10.0, 11 * 10.0, 0.0] for x in range(3, NX - 3, 5)])
    om, g = _models(NX, NY, NZ, prec, p=p, max_receivers=len(rec))
    sx, sy, sz = 21 * 10.0 + 3.0, 12 * 10.0 - 4.0, 3 * 10.0
    src = W.PointSource3D(om, sx, sy, sz, 25.0, 0.05, amp=1e3, p=p)
    si, ri = g.set_source_receivers3d(0, sx, sy, sz, 25.0, 0.05, 1e3, rec)
    assert (si[2], si[1], si[0]) == src.node
    rn = W.receiver_nodes3d(om, rec)
    assert np.array_equal(ri[:, ::-1], rn)                  # integer indices: bit-exact
    U0 = tuple(smooth_random_state(om.field_shapes(), 8))
    return om, g, src, rec, rn, U0


def _oracle_steps(om, method, U0, src, t, dt, m, nsteps, rn):
    params = faber.ellipse_params(om.c_max, om.beta0, om.dx, om.order, dims=3,
                                  free_surface=om.free_surface)
    U, S = U0, []
    if method == "leapfrog":
        LF = PML.leapfrog3dp_init(U0)
    for n in range(nsteps):
        tn = t + n * dt
        if method == "faber":
            U = faber.faber_step(om, U, src, tn, dt, m, params)
        elif method == "krylov":
            U = krylov.krylov_step(om, U, src, tn, dt, m)
        elif method == "hork":
            U = rk.hork_step(om, U, src, tn, dt, m)
        elif method == "rk32":
            U = rk.rk32_step(om, U, src, tn, dt)
        elif method == "rk44":
            U = rk.rk44_step(om, U, src, tn, dt)
        elif method == "leapfrog":
            LF = PML.leapfrog3dp_step(om, LF, src, tn, dt)
            U = (LF[0], U[1], LF[2], LF[4], LF[6], LF[8])
        S.append(U[0][rn[:, 0], rn[:, 1], rn[:, 2]].copy())
    return U, np.array(S)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("method,m", [("faber", 14), ("krylov", 10), ("hork", 6), ("rk32", 0),
                                      ("rk44", 0), ("leapfrog", 0), ("faber", 1), ("hork", 1),
                                      ("hork-horner", 6), ("hork-horner", 1)])
def test_integrators_match_oracle_3d(prec, method, m):
    """m = 1 covers the copy of a work vector into the state (all six fields)."""
    om, g, src, rec, rn, U0 = _setup(prec)
    if method == "hork-horner":
        g.set_hork_form("horner")
        method = "hork"
    if method in ("krylov", "leapfrog"):
        # displacement at rest (Krylov conditioning; leap-frog starts from u^{-1} = u^0)
        U0 = (U0[0],) + tuple(0 * f for f in U0[1:])
    dt = 3e-4 if method == "leapfrog" else 1.0e-3
    t, nsteps = 0.03, 3
    if method == "faber":
        g.set_faber_ellipse(*faber.ellipse_params(om.c_max, om.beta0, om.dx, 8, dims=3,
                                                  free_surface=True))
    g.bind_seismogram(nsteps)
    g.set_state(0, flatten(U0))
    g.step(method, t, dt, m, nsteps)
    got = g.get_state(0)
    U, S = _oracle_steps(om, method, U0, src, t, dt, m, nsteps, rn)
    if method == "leapfrog":     # v is not advanced by leap-frog: compare u and the w fields
        sizes = [int(np.prod(s)) for s in om.field_shapes()]
        keep = np.concatenate([np.ones(sizes[0], bool), np.zeros(sizes[1], bool),
                               np.ones(sum(sizes[2:]), bool)])
        got, ref = got[keep], flatten(U)[keep]
    else:
        ref = flatten(U)
    tol = TOL[prec] * (3 if prec == "f32" else 1)
    assert rel_l2(got, ref) < tol, (method, m, rel_l2(got, ref))
    shapes = om.field_shapes()
    if method == "leapfrog":
        shapes = [shapes[0]] + shapes[2:]
    per_field = rel_l2_fields(got, ref, shapes)
    assert max(per_field) < tol, (method, m, per_field)
    Sg = g.seismogram(0, len(rec), nsteps)
    assert rel_l2(Sg, S) < tol
    g.close()


def test_default_ellipse_is_the_3d_one():
    om, g = _models(30, 20, 25, "f64", fs=True)
    want = faber.ellipse_params(om.c_max, om.beta0, om.dx, 8, dims=3, free_surface=True)
    assert np.allclose(g.faber_ellipse(), want, rtol=1e-12)
    g.close()


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("method,m", [("faber", 12), ("hork", 5), ("rk44", 0), ("leapfrog", 0)])
def test_fp32_pass_variants_match_oracle_3d(variant, method, m):
    """FP32 3D passes: variants 0 and 2 are the persistent TMA pipeline (64 x 8 column tiles,
    z chunks of 32 planes, warm-up stages) with 16 and 8 consumer warps, variant 1 the plain
    z-marching kernel.  NZ = 38 spans two chunks and the free-surface planes; NX, NY are
    ragged."""
    om, g, src, rec, rn, U0 = _setup("f32")
    g.set_kernel_variant(variant)
    dt, t, nsteps = (3e-4 if method == "leapfrog" else 1.0e-3), 0.03, 2
    if method == "faber":
        g.set_faber_ellipse(*faber.ellipse_params(om.c_max, om.beta0, om.dx, 8, dims=3,
                                                  free_surface=True))
    g.bind_seismogram(nsteps)
    g.set_state(0, flatten(U0))
    g.step(method, t, dt, m, nsteps)
    U, S = _oracle_steps(om, method, U0, src, t, dt, m, nsteps, rn)
    got = g.get_state(0)
    assert rel_l2(got, flatten(U)) < 3 * TOL["f32"]
    assert max(rel_l2_fields(got, flatten(U), om.field_shapes())) < 3 * TOL["f32"]
    assert rel_l2(g.seismogram(0, len(rec), nsteps), S) < 3 * TOL["f32"]
    g.close()

"""Pins of the auxiliary-field 3D PML oracle (oracle/wave3d_pml.py): two independent routes,
exact reduction to Eq. 1 with damping on a field that does not vary along an undamped axis,
reduction to the 3D operator without damping, and a stable dense spectrum."""
import numpy as np
import pytest

from oracle import operator as O
from oracle import wave3d as W
from oracle import wave3d_pml as P
from oracle.model import Model, default_beta0, flatten, unflatten
from paper_2401_16322_gb300.workloads import layered, layered3d, smooth_random_state


def _m3(nx=10, ny=9, nz=11, pml=3, fs=True, order=8, beta=True, seed=6):
    c = layered3d(nx, ny, nz, seed, vmin=1500, vmax=3000)
    b0 = default_beta0(3000.0, pml, 10.0) if beta else 0.0
    return W.Model3D(nx, ny, nz, 10.0, order, pml, b0, fs, c)


def _split(m, x):
    out, o = [], 0
    for s in P.field_shapes(m):
        n = int(np.prod(s))
        out.append(x[o:o + n].reshape(s))
        o += n
    return tuple(out)


@pytest.mark.parametrize("fs,order,undamped", [(True, 8, ()), (False, 8, ()), (False, 4, ()),
                                               (True, 8, ("y",))])
def test_matrix_free_equals_assembled(fs, order, undamped):
    m = _m3(fs=fs, order=order)
    x = flatten(smooth_random_state(P.field_shapes(m), 3))
    a = flatten(P.apply_H3p(m, _split(m, x), undamped=undamped))
    b = P.assemble_H3p(m, undamped=undamped) @ x
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_reduces_to_eq1_with_damping_on_a_y_invariant_field():
    """No damping along y and a field constant in y (w_y = 0): on the y rows at least R from
    the y edges, the v, w_x and w_z rows equal Eq. 1's 2D operator on the x-z slice with its
    damping and free-surface rows; w_y stays zero and psi_t = u."""
    nx, ny, nz, pml = 13, 11, 12, 3
    c2d = layered(nx, nz, 7, vmin=1500, vmax=3000)
    b0 = default_beta0(3000.0, pml, 10.0)
    c3 = np.repeat(c2d[:, None, :], ny, axis=1)
    m3 = W.Model3D(nx, ny, nz, 10.0, 8, pml, b0, True, c3)
    m2 = Model(nx, nz, 10.0, 8, pml, b0, True, c2d)
    u2, v2, wx2, wz2 = smooth_random_state(m2.field_shapes(), 21)
    psi = np.repeat(smooth_random_state([(nz, nx)], 22)[0][:, None, :], ny, 1)   # y-invariant
    U3 = (np.repeat(u2[:, None, :], ny, 1), np.repeat(v2[:, None, :], ny, 1),
          np.repeat(wx2[:, None, :], ny, 1), np.zeros((nz, ny - 1, nx)),
          np.repeat(wz2[:, None, :], ny, 1), psi)
    h3 = P.apply_H3p(m3, U3, undamped=("y",))
    h2 = O.apply_H(m2, (u2, v2, wx2, wz2))
    for j in range(4, ny - 4):
        for got, ref in ((h3[1][:, j, :], h2[1]), (h3[2][:, j, :], h2[2]), (h3[4][:, j, :], h2[3])):
            assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.max(np.abs(ref)))
    assert np.array_equal(h3[0], U3[1]) and np.array_equal(h3[5], U3[0])
    assert np.max(np.abs(h3[3][:, 4:ny - 5, :])) == 0.0


def test_mean_reading_does_not_reduce_where_this_one_does():
    """The same y-invariant comparison against oracle.wave3d's mean-of-the-others reading
    fails in the damped layer: the reason this formulation exists."""
    nx, ny, nz, pml = 13, 11, 12, 3
    c2d = layered(nx, nz, 7, vmin=1500, vmax=3000)
    b0 = default_beta0(3000.0, pml, 10.0)
    m3 = W.Model3D(nx, ny, nz, 10.0, 8, pml, b0, True, np.repeat(c2d[:, None, :], ny, axis=1))
    m2 = Model(nx, nz, 10.0, 8, pml, b0, True, c2d)
    u2, v2, wx2, wz2 = smooth_random_state(m2.field_shapes(), 21)
    U3 = (np.repeat(u2[:, None, :], ny, 1), np.repeat(v2[:, None, :], ny, 1),
          np.repeat(wx2[:, None, :], ny, 1), np.zeros((nz, ny - 1, nx)),
          np.repeat(wz2[:, None, :], ny, 1))
    h2 = O.apply_H(m2, (u2, v2, wx2, wz2))
    h3 = W.apply_H3(m3, U3)
    j = ny // 2                                   # interior in y: beta_y = 0 there
    assert not np.allclose(h3[2][:, j, :], h2[2], rtol=1e-6, atol=1e-6 * np.max(np.abs(h2[2])))


def test_without_damping_equals_the_3d_operator():
    m = _m3(beta=False)
    U = tuple(smooth_random_state(P.field_shapes(m), 4))
    hp = P.apply_H3p(m, U)
    h = W.apply_H3(m, U[:5])
    for a, b in zip(hp[:5], h):
        assert np.allclose(a, b, rtol=1e-14, atol=1e-14 * np.max(np.abs(b)))
    assert np.array_equal(hp[5], U[0])


def test_dense_spectrum_is_stable():
    """No growing mode: on a small free-surface cube the largest real part of the dense
    spectrum is at round-off level (2e-13 against beta0 = 1036 s^-1), while the damped modes
    reach Re(lambda) = -529 s^-1."""
    m = _m3(nx=8, ny=7, nz=8, pml=3)
    ev = np.linalg.eigvals(P.assemble_H3p(m).toarray())
    assert ev.real.max() < 1e-9 * m.beta0
    assert ev.real.min() < -0.1 * m.beta0

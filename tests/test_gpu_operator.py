"""GPU parity of the operator H (Eq. 1) and its transpose against the oracle, through the
C ABI.  Grids span several 64 x 16 tiles with ragged tails."""
import numpy as np
import pytest

from _helpers import TOL, flatten, gpu_model, oracle_model, rel_l2, unflatten
from oracle.operator import apply_H, assemble_H
from paper_2401_16322_gb300.workloads import layered, random_state, smooth_random_state

pytestmark = pytest.mark.gpu

CASES = [
    # (nx, ny, order, fs, pml)
    (137, 53, 8, True, 12),
    (70, 35, 8, False, 9),
    (101, 41, 4, False, 20),
    (12, 10, 8, True, 4),       # smaller than one tile
    (65, 17, 8, True, 0),       # one column / one row into the next tile, no damping
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny,order,fs,pml", CASES)
def test_apply_H_matches_oracle(prec, nx, ny, order, fs, pml):
    c = layered(nx, ny, 7)
    om = oracle_model(nx, ny, c, order=order, pml=pml, fs=fs)
    g = gpu_model(om, prec)
    for seed, gen in ((1, smooth_random_state), (2, random_state)):
        U = gen([f.shape for f in om.zeros_state()], seed)
        x = flatten(U)
        ref = flatten(apply_H(om, unflatten(om, x)))
        got = g.apply(x)
        assert rel_l2(got, ref) < TOL[prec], (prec, seed, rel_l2(got, ref))


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny,order,fs,pml", CASES[:3] + CASES[3:4])
def test_apply_HT_matches_assembled_transpose(prec, nx, ny, order, fs, pml):
    c = layered(nx, ny, 8)
    om = oracle_model(nx, ny, c, order=order, pml=pml, fs=fs)
    HT = assemble_H(om).T.tocsr()
    g = gpu_model(om, prec)
    y = flatten(random_state([f.shape for f in om.zeros_state()], 5))
    ref = HT @ y
    got = g.apply(y, transpose=True)
    assert rel_l2(got, ref) < TOL[prec], rel_l2(got, ref)


def test_adjoint_identity_on_gpu():
    """<H x, y> = <x, H^T y> with both products from the GPU kernels (FP64)."""
    nx, ny = 90, 44
    om = oracle_model(nx, ny, layered(nx, ny, 3), pml=10, fs=True)
    g = gpu_model(om, "f64")
    x, y = (flatten(random_state([f.shape for f in om.zeros_state()], s)) for s in (11, 12))
    lhs = float(np.dot(g.apply(x), y))
    rhs = float(np.dot(x, g.apply(y, transpose=True)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_padding_stays_zero():
    """Pad columns/rows of the padded layout are written as zeros."""
    import torch
    nx, ny = 37, 21
    om = oracle_model(nx, ny, layered(nx, ny, 1), pml=5, fs=True)
    g = gpu_model(om, "f32")
    x = g.new_vector()
    g.pack(flatten(random_state([f.shape for f in om.zeros_state()], 3)), x)
    y = g.new_vector().fill_(7.0)
    g.apply_device(x, y)
    torch.cuda.synchronize()
    P = g.layout.pitch
    Y = y.view(4, ny, P).cpu().numpy()
    assert np.all(Y[:, :, nx:] == 7.0)          # never touched beyond nx
    assert np.all(Y[2, :, nx - 1] == 0.0)       # w_x pad column
    assert np.all(Y[3, ny - 1, :nx] == 0.0)     # w_y pad row

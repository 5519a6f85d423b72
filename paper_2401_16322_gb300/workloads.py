"""Seeded synthetic inputs (velocity models and acquisition geometry).

This module is shared by the CUDA path's tests/benchmarks and by the CPU oracle's tests.  It
holds none of the method's arithmetic: it only draws velocity models and source/receiver
positions (in metres).  The paper's velocity models (Corner, Santos Basin, Marmousi,
SEG/EAGE; Sec. 5.1) are not available, so layered models with smooth random perturbations
of the same grid spacing (dx = 10 m) and velocity range stand in for them.

Recipes (all with numpy's PCG64 generator):

* ``layered``: ``n_interfaces`` interface depths drawn uniformly and sorted; layer velocities
  rise linearly from ``vmin`` to ``vmax`` with +-``jitter`` relative uniform jitter; an
  N(0, 1) field smoothed by a Gaussian of ``sigma_cells`` cells, normalised to unit
  standard deviation and scaled by ``pert`` * c is added; the result is clipped to
  [vmin, vmax].
* ``smooth_gradient_with_anomalies``: v(z) = v0 + k z smoothed, plus three Gaussian
  anomalies (+10 %, -10 %, +10 %) of ``sigma_cells`` cells at seeded interior positions.
* ``homogeneous``: constant velocity.
"""
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np
from scipy.ndimage import gaussian_filter


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def homogeneous(nx, ny, c):
    return np.full((ny, nx), float(c))


def layered(nx, ny, seed, vmin=1500.0, vmax=4500.0, n_interfaces=8, jitter=0.05,
            sigma_cells=8.0, pert=0.05):
    rng = _rng(seed)
    depths = np.sort(rng.uniform(0.0, ny, size=n_interfaces))
    nl = n_interfaces + 1
    base = np.linspace(vmin, vmax, nl) * (1.0 + jitter * rng.uniform(-1.0, 1.0, size=nl))
    j = np.arange(ny)[:, None] + 0.5
    layer = np.searchsorted(depths, j[:, 0])
    c = np.repeat(base[layer][:, None], nx, axis=1)
    noise = gaussian_filter(rng.standard_normal((ny, nx)), sigma_cells, mode="reflect")
    noise /= max(noise.std(), 1e-30)
    c = c + pert * c * noise
    return np.clip(c, vmin, vmax)


def smooth_gradient_with_anomalies(nx, ny, seed, dx=10.0, v0=1800.0, k=1.2, sigma_cells=15.0,
                                   margin=0, amps=(0.10, -0.10, 0.10), smooth_cells=4.0):
    rng = _rng(seed)
    z = (np.arange(ny)[:, None] * dx) * np.ones((1, nx))
    c = gaussian_filter(v0 + k * z, smooth_cells, mode="nearest")
    jj, ii = np.mgrid[0:ny, 0:nx]
    lo_i, hi_i = margin + 2 * sigma_cells, nx - margin - 2 * sigma_cells
    lo_j, hi_j = 2 * sigma_cells, ny - margin - 2 * sigma_cells
    for a in amps:
        ci = rng.uniform(lo_i, max(hi_i, lo_i + 1))
        cj = rng.uniform(lo_j, max(hi_j, lo_j + 1))
        c = c * (1.0 + a * np.exp(-((ii - ci) ** 2 + (jj - cj) ** 2) / (2 * sigma_cells ** 2)))
    return c


@dataclass
class Shot:
    """One source (metres; y is depth below the top row) and its receivers."""
    sx: float
    sy: float
    rec: np.ndarray            # (nrec, 2) metres, columns (x, depth)


@dataclass
class Workload:
    """A model with its acquisition; the numeric parameters of the method ride along."""
    name: str
    nx: int
    ny: int
    dx: float
    order: int
    pml: int
    free_surface: bool
    c: np.ndarray = field(repr=False)
    shots: List[Shot] = field(default_factory=list)
    f_peak: float = 10.0
    T: float = 1.0


def t0_for(f_peak):
    """Source delay: 0.18 s at 15 Hz generalised to 2.7 / f_peak."""
    return 2.7 / f_peak


def config_homogeneous_small():
    """101 x 101, dx 10 m, c 2000 m/s, 4th order, 20-point ABC on all sides (no free
    surface), Ricker 15 Hz at the centre, 50 receivers on row 25, columns 25..74, T 0.5 s."""
    nx = ny = 101
    dx = 10.0
    rec = np.array([[i * dx, 25 * dx] for i in range(25, 75)])
    return Workload("homogeneous-101x101-o4", nx, ny, dx, 4, 20, False, homogeneous(nx, ny, 2000.0),
                    [Shot(50 * dx, 50 * dx, rec)], f_peak=15.0, T=0.5)


def config_layered_601x301(seed=2401):
    """601 x 301 layered model, 8th order, 40-point ABC, free surface, Ricker 10 Hz at
    (300, 2), receivers on row 0 every 2nd column, T 2 s."""
    nx, ny, dx = 601, 301, 10.0
    rec = np.array([[i * dx, 0.0] for i in range(0, nx, 2)])
    return Workload("layered-601x301-o8", nx, ny, dx, 8, 40, True, layered(nx, ny, seed),
                    [Shot(300 * dx, 2 * dx, rec)], f_peak=10.0, T=2.0)


def config_batched(seed=2401, nshots=64):
    """One 1001 x 501 layered model with ``nshots`` sources on row 2 at columns 40 + 14 k,
    plus eight models with sizes linearly spaced from 201 x 101 to 801 x 401, each with one
    centre-surface shot.  8th order, 40-point ABC, free surface, Ricker 10 Hz."""
    dx = 10.0
    out = []
    nx, ny = 1001, 501
    rec = np.array([[i * dx, 0.0] for i in range(0, nx, 4)])
    shots = [Shot((40 + 14 * k) * dx, 2 * dx, rec) for k in range(nshots)]
    out.append(Workload("layered-1001x501-o8", nx, ny, dx, 8, 40, True, layered(nx, ny, seed),
                        shots, f_peak=10.0, T=2.0))
    sizes = [(int(round(201 + (801 - 201) * q / 7)), int(round(101 + (401 - 101) * q / 7)))
             for q in range(8)]
    for q, (mx, my) in enumerate(sizes):
        recq = np.array([[i * dx, 0.0] for i in range(0, mx, 4)])
        out.append(Workload(f"layered-{mx}x{my}-o8", mx, my, dx, 8, 40, True,
                            layered(mx, my, seed + 1 + q), [Shot((mx // 2) * dx, 2 * dx, recq)],
                            f_peak=10.0, T=2.0))
    return out


def config_fwi(seed=2402, nshots=16):
    """401 x 201 smooth v(z) = 1800 + 1.2 z background with three +-10 % Gaussian
    anomalies, 16 shots evenly along row 2, 200 receivers on row 0, T 1.5 s."""
    nx, ny, dx = 401, 201, 10.0
    c = smooth_gradient_with_anomalies(nx, ny, seed, dx=dx, margin=40)
    rec = np.array([[x, 0.0] for x in np.linspace(0.0, (nx - 1) * dx, 200)])
    xs = np.linspace(40 * dx, (nx - 41) * dx, nshots)
    shots = [Shot(float(x), 2 * dx, rec) for x in xs]
    return Workload("fwi-401x201-o8", nx, ny, dx, 8, 40, True, c, shots, f_peak=10.0, T=1.5)


def layered3d(nx, ny, nz, seed, vmin=1500.0, vmax=4500.0, n_interfaces=8, jitter=0.05,
              sigma_cells=8.0, pert=0.05):
    """The layered model of ``layered`` with the layers along z (depth, the slowest axis):
    velocity c[k, j, i], interfaces at sorted uniform depths, rising layer velocities with
    jitter, plus Gaussian-smoothed noise (unit std, x pert) clipped to [vmin, vmax]."""
    rng = _rng(seed)
    depths = np.sort(rng.uniform(0.0, nz, size=n_interfaces))
    nl = n_interfaces + 1
    base = np.linspace(vmin, vmax, nl) * (1.0 + jitter * rng.uniform(-1.0, 1.0, size=nl))
    layer = np.searchsorted(depths, np.arange(nz) + 0.5)
    c = np.broadcast_to(base[layer][:, None, None], (nz, ny, nx)).astype(np.float64)
    noise = gaussian_filter(rng.standard_normal((nz, ny, nx)).astype(np.float32), sigma_cells,
                            mode="reflect").astype(np.float64)
    noise /= max(noise.std(), 1e-30)
    c = c + pert * c * noise
    return np.clip(c, vmin, vmax)


@dataclass
class Workload3D:
    """One three-dimensional model with a single shot (positions in metres, z = depth)."""
    name: str
    n: int
    dx: float
    order: int
    pml: int
    free_surface: bool
    c: np.ndarray            # [nz, ny, nx]
    src: Tuple[float, float, float]
    rec: np.ndarray          # [nrec, 3] (x, y, depth)
    f_peak: float
    T: float


def config_3d(n=400, seed=2403, pml=30, T=1.0):
    """n^3 layered model (layers along depth, as ``layered``), dx 10 m, 8th order, free
    surface, ``pml``-point ABC, Ricker 10 Hz at the centre two cells below the surface,
    receivers every 4th node along the centre line of the surface, T 1 s."""
    dx = 10.0
    c = layered3d(n, n, n, seed)
    mid = (n // 2) * dx
    rec = np.array([[i * dx, mid, 0.0] for i in range(0, n, 4)])
    return Workload3D(f"layered3d-{n}^3-o8", n, dx, 8, pml, True, c, (mid, mid, 2 * dx), rec,
                      10.0, T)


def random_state(shape_list: List[Tuple[int, ...]], seed, scale=1.0):
    """Seeded N(0, scale^2) arrays of the given shapes (test inputs for operator parity)."""
    rng = _rng(seed)
    return [scale * rng.standard_normal(s) for s in shape_list]


def smooth_random_state(shape_list: List[Tuple[int, ...]], seed, sigma_cells=3.0):
    """Seeded smooth fields (Gaussian-filtered noise, unit std) of the given shapes."""
    rng = _rng(seed)
    out = []
    for s in shape_list:
        a = gaussian_filter(rng.standard_normal(s), sigma_cells)
        out.append(a / max(a.std(), 1e-30))
    return out

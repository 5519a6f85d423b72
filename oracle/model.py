"""Model description and the PML damping profile of the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Grid (Sec. 2.1, Fig. 1): u, v and c live on the nodes (i, j), i = 0..nx-1 (x to the right),
j = 0..ny-1 (j = 0 is the top row; depth y = -j dx grows with j); w_x on the half points
(i+1/2, j), i = 0..nx-2; w_y on (i, j+1/2), j = 0..ny-2.  Values beyond these index ranges
are zero (the zero extension of Sec. 2.1).

Damping (Sec. 2, the beta_z formula): beta_z = beta0 (1 - d/delta)^2 where the distance d
to the boundary is at most delta (= pml_width * dx), else 0.  Reading of the unstated
geometry: the boundary lies on the first ghost line outside the unknowns (i = -1, i = nx,
j = ny, and j = -1 when there is no free surface), so a node at i has d = min(i+1, nx-i) dx
and a half point at i+1/2 has d = min(i+3/2, nx-i-1/2) dx.  With a free surface the top
strip has no PML, so beta_y depends on the bottom distance only.  beta is evaluated at the
location of the variable being updated.

Parity status: pinned indirectly (energy conservation at beta0 = 0 and the dense
exponential checks use this module); the profile formula itself is "parity unpinned"
beyond the closed-form spot values of tests/test_oracle_operator.py
(``test_damping_profile_values``).
"""
from dataclasses import dataclass, field
import math

import numpy as np


def default_beta0(c_max, pml_width, dx, reflection=1e-3):
    """Common quadratic-profile choice beta0 = 3 c_max / (2 delta) ln(1/R) (beta0 is unstated)."""
    if pml_width <= 0:
        return 0.0
    delta = pml_width * dx
    return 3.0 * c_max / (2.0 * delta) * math.log(1.0 / reflection)


@dataclass
class Model:
    nx: int
    ny: int
    dx: float
    order: int           # 4 or 8
    pml: int             # PML width in grid points (delta = pml * dx)
    beta0: float
    free_surface: bool
    c: np.ndarray = field(repr=False)   # velocity at nodes, shape (ny, nx)

    def __post_init__(self):
        self.c = np.asarray(self.c, dtype=np.float64)
        if self.c.shape != (self.ny, self.nx):
            raise ValueError("c must have shape (ny, nx)")
        if self.order not in (4, 8):
            raise ValueError("order must be 4 or 8")
        if self.free_surface and self.order != 8:
            raise ValueError("free-surface rows exist for 8th order only")
        if self.nx < 2 or self.ny < 2:
            raise ValueError("grid must be at least 2 x 2")

    @property
    def c2(self):
        return self.c * self.c

    @property
    def c_max(self):
        return float(self.c.max())

    # -- damping ---------------------------------------------------------------------
    def _beta(self, d):
        """beta0 (1 - d/delta)^2 for d <= delta, d and delta in grid units."""
        d = np.asarray(d, dtype=np.float64)
        if self.pml <= 0:
            return np.zeros_like(d)
        return np.where(d <= self.pml, self.beta0 * (1.0 - d / self.pml) ** 2, 0.0)

    def beta_x_node(self):
        i = np.arange(self.nx, dtype=np.float64)
        return self._beta(np.minimum(i + 1.0, self.nx - i))

    def beta_x_half(self):
        i = np.arange(self.nx - 1, dtype=np.float64)
        return self._beta(np.minimum(i + 1.5, self.nx - i - 0.5))

    def beta_y_node(self):
        j = np.arange(self.ny, dtype=np.float64)
        d = (self.ny - j) if self.free_surface else np.minimum(j + 1.0, self.ny - j)
        return self._beta(d)

    def beta_y_half(self):
        j = np.arange(self.ny - 1, dtype=np.float64)
        d = (self.ny - j - 0.5) if self.free_surface else np.minimum(j + 1.5, self.ny - j - 0.5)
        return self._beta(d)

    # -- sizes -----------------------------------------------------------------------
    @property
    def n(self):
        """Length of the state vector (u, v, w_x, w_y)."""
        return 2 * self.nx * self.ny + (self.nx - 1) * self.ny + self.nx * (self.ny - 1)

    def field_shapes(self):
        nx, ny = self.nx, self.ny
        return [(ny, nx), (ny, nx), (ny, nx - 1), (ny - 1, nx)]

    def zeros_state(self):
        return tuple(np.zeros(s) for s in self.field_shapes())


def flatten(state):
    """(u, v, w_x, w_y) -> one vector in that order (row-major fields)."""
    return np.concatenate([np.ravel(f) for f in state])


def unflatten(model, x):
    """Inverse of ``flatten`` for the model's field shapes (2D: u, v, w_x, w_y; 3D adds w_z)."""
    out, o = [], 0
    for sh in model.field_shapes():
        s = int(np.prod(sh))
        out.append(np.asarray(x[o:o + s], dtype=np.float64).reshape(sh))
        o += s
    return tuple(out)

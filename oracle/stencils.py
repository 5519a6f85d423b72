"""Finite-difference stencil tables of the oracle (exact rationals, converted to FP64 on use).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sources in the paper (arXiv 2401.16322):

* Sec. 2.1, Eq. (spatial_8th_1): 8th-order staggered first derivative
  (1225/(1024 dx)) [(u_{i+1}-u_i) - (u_{i+2}-u_{i-1})/15 + (u_{i+3}-u_{i-2})/125
  - (u_{i+4}-u_{i-3})/1715].  Used as printed.
* Sec. 2.1, Eq. (spatial_8th_2): 8th-order centred second derivative.  Read with "+" between
  the symmetric pairs and over dx^2 (the printed "-" would make the stencil odd and
  inconsistent; with "+" the weights sum to 0 and the second moment is 2).
* Appendix A: one-sided u_yy rows at y = 0, -dx, -2dx, -3dx and u_y rows at y = -dx/2,
  -3dx/2, -5dx/2, in the physical coordinate y (upward), with u_i = u(x, -i dx).
* Sec. 2.2: d(w_y)/dy at the first four node rows by Fornberg's algorithm on the points
  y = 0 (where w_y = 0 at the free surface) and the eight nearest half rows.
* 4th-order tables (not in the paper, which is 8th order only): Fornberg weights on the
  symmetric 4-point staggered and 5-point centred sets.

Pins (tests/test_oracle_stencils.py): moments of every table against exact monomial
derivatives; Fornberg reproduces the printed interior stencils; the Appendix A rows are
re-derived by an exact Vandermonde solve.
"""
from fractions import Fraction as Fr

import numpy as np


def fornberg_weights(z, x, m):
    """Fornberg (1988) weights for derivatives 0..m at ``z`` from values at points ``x``.

    Returns ``C`` with ``C[k][j]`` the weight of point ``x[j]`` in the k-th derivative.
    Works for any field type (``Fraction`` for exact weights, ``float``).  The algorithm
    builds the weights for the point sets x[0..i] one point at a time, updating the old
    points' weights and creating the new point's weights from the previous set.
    """
    n = len(x)
    one = x[0] * 0 + 1
    zero = one * 0
    C = [[zero] * n for _ in range(m + 1)]
    C[0][0] = one
    c1 = one
    c4 = x[0] - z
    for i in range(1, n):
        mn = min(i, m)
        c2 = one
        c5 = c4
        c4 = x[i] - z
        for j in range(i):
            c3 = x[i] - x[j]
            c2 = c2 * c3
            if j == i - 1:
                for k in range(mn, 0, -1):
                    C[k][i] = c1 * (k * C[k - 1][i - 1] - c5 * C[k][i - 1]) / c2
                C[0][i] = -c1 * c5 * C[0][i - 1] / c2
            for k in range(mn, 0, -1):
                C[k][j] = (c4 * C[k][j] - k * C[k - 1][j]) / c3
            C[0][j] = c4 * C[0][j] / c3
        c1 = c2
    return C


# ---------------------------------------------------------------------------------------
# Interior stencils.  STAG[R][k] multiplies (u_{i+1+k} - u_{i-k}) for the derivative at the
# half point i+1/2; CENT[R][k] multiplies (u_{i+k} + u_{i-k}) (k >= 1) and u_i (k = 0).
# ---------------------------------------------------------------------------------------

# Eq. (spatial_8th_1), as printed: 1225/1024 * [1, -1/15, 1/125, -1/1715].
STAG8 = [Fr(1225, 1024) * f for f in (Fr(1), Fr(-1, 15), Fr(1, 125), Fr(-1, 1715))]
# Eq. (spatial_8th_2), read with "+" between symmetric pairs.
CENT8 = [Fr(-205, 72), Fr(8, 5), Fr(-1, 5), Fr(8, 315), Fr(-1, 560)]


def _fornberg_staggered(R):
    pts = [Fr(2 * k + 1, 2) for k in range(-R, R)]  # offsets of u_{i-R+1}..u_{i+R} from i+1/2
    w = fornberg_weights(Fr(0), pts, 1)[1]
    # weight of u_{i+1+k} sits at index R+k; of u_{i-k} at index R-1-k
    return [w[R + k] for k in range(R)]


def _fornberg_centred(R):
    pts = [Fr(k) for k in range(-R, R + 1)]
    w = fornberg_weights(Fr(0), pts, 2)[2]
    return [w[R + k] for k in range(R + 1)]


STAG4 = _fornberg_staggered(2)   # [9/8, -1/24]
CENT4 = _fornberg_centred(2)     # [-5/2, 4/3, -1/12]

STAG = {8: STAG8, 4: STAG4}
CENT = {8: CENT8, 4: CENT4}


def half_width(order):
    """Stencil half-width R (4 for 8th order, 2 for 4th order)."""
    if order not in (4, 8):
        raise ValueError("fd order must be 4 or 8")
    return order // 2


# ---------------------------------------------------------------------------------------
# Appendix A: free-surface rows, physical y, u_i = u(x, -i dx).
# ---------------------------------------------------------------------------------------
FS_UYY = [
    [Fr(-3144919, 352800), Fr(16), Fr(-14), Fr(112, 9), Fr(-35, 4), Fr(112, 25), Fr(-14, 9),
     Fr(16, 49), Fr(-1, 32)],
    [Fr(271343, 156800), Fr(-1991, 630), Fr(57, 40), Fr(13, 60), Fr(-109, 288), Fr(6, 25),
     Fr(-11, 120), Fr(179, 8820), Fr(-9, 4480)],
    [Fr(-18519, 78400), Fr(58, 35), Fr(-251, 90), Fr(22, 15), Fr(-1, 16), Fr(-14, 225),
     Fr(1, 30), Fr(-2, 245), Fr(17, 20160)],
    [Fr(74801, 1411200), Fr(-37, 140), Fr(67, 40), Fr(-263, 90), Fr(53, 32), Fr(-23, 100),
     Fr(13, 360), Fr(-1, 245), Fr(1, 4480)],
]
FS_UY = [
    [Fr(5034629, 3763200), Fr(-23533, 15360), Fr(4259, 15360), Fr(-1103, 9216), Fr(151, 3072),
     Fr(-1171, 76800), Fr(139, 46080), Fr(-211, 752640)],
    [Fr(-363509, 3763200), Fr(6297, 5120), Fr(-6147, 5120), Fr(211, 3072), Fr(3, 1024),
     Fr(-153, 25600), Fr(29, 15360), Fr(-57, 250880)],
    [Fr(4631, 250880), Fr(-305, 3072), Fr(1245, 1024), Fr(-3725, 3072), Fr(275, 3072),
     Fr(-69, 5120), Fr(5, 3072), Fr(-5, 50176)],
]


def fs_dwy_weights():
    """Sec. 2.2: d(w_y)/dy at node rows j = 0..3 (y = -j dx), 8th order, by Fornberg.

    Points: y = 0, where w_y = 0 (free surface), and the half rows y = -(q+1/2) dx,
    q = 0..7, holding w_y[q].  Returns a 4 x 8 table of weights on w_y[0..7] (units 1/dx);
    the weight of the y = 0 point multiplies a known zero and is dropped.
    """
    pts = [Fr(0)] + [-Fr(2 * q + 1, 2) for q in range(8)]
    rows = []
    for j in range(4):
        w = fornberg_weights(Fr(-j), pts, 1)[1]
        rows.append(w[1:])
    return rows


FS_DWY = fs_dwy_weights()

N_FS_UYY_ROWS = 4   # node rows 0..3 replaced for u_yy and d(w_y)/dy
N_FS_UY_ROWS = 3    # half rows 0..2 replaced for u_y


def as_float(table):
    """Convert a (nested) list of Fractions to a float64 numpy array."""
    return np.array([[float(c) for c in row] for row in table]) if isinstance(table[0], list) \
        else np.array([float(c) for c in table])

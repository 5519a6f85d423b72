"""Pins of the oracle's stencil tables (Sec. 2.1, Sec. 2.2, Appendix A) against exact
mathematics: monomial moments, an independent exact Vandermonde solve, and the golden file
of the paper's printed rationals."""
import os
from fractions import Fraction as Fr

import pytest

from oracle import stencils as S


def _golden(repo_root):
    rows = {}
    with open(os.path.join(repo_root, "tests", "golden", "stencils_printed.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows[key] = [Fr(v) for v in vals]
    return rows


def test_oracle_tables_match_printed_values(repo_root):
    g = _golden(repo_root)
    assert S.STAG8 == g["stag8"]
    assert S.CENT8 == g["cent8"]
    for r in range(4):
        assert S.FS_UYY[r] == g[f"uyy{r}"]
    for r in range(3):
        assert S.FS_UY[r] == g[f"uy{r}"]


@pytest.mark.parametrize("R", [2, 4])
def test_staggered_moments(R):
    """sum_k s_k ((k+1/2)^q - (-(k+1/2))^q) = [q == 1] for q <= 2R, and fails at q = 2R+1."""
    s = S.STAG[2 * R]
    for q in range(0, 2 * R + 2):
        mom = sum(s[k] * (Fr(2 * k + 1, 2) ** q - Fr(-(2 * k + 1), 2) ** q) for k in range(R))
        if q <= 2 * R:
            assert mom == (1 if q == 1 else 0), q
        else:
            assert mom != 0


@pytest.mark.parametrize("R", [2, 4])
def test_centred_moments(R):
    """d_0 [q == 0] + sum_k d_k (k^q + (-k)^q) = 2 [q == 2] for q <= 2R+1; fails at 2R+2."""
    d = S.CENT[2 * R]
    for q in range(0, 2 * R + 3):
        mom = (d[0] if q == 0 else 0) + sum(d[k] * (Fr(k) ** q + Fr(-k) ** q)
                                            for k in range(1, R + 1))
        if q <= 2 * R + 1:
            assert mom == (2 if q == 2 else 0), q
        else:
            assert mom != 0


def test_fornberg_reproduces_paper_interior():
    assert S._fornberg_staggered(4) == S.STAG8
    assert S._fornberg_centred(4) == S.CENT8


def test_fourth_order_textbook_values():
    # 4th-order staggered (9/8, -1/24) and centred (-5/2, 4/3, -1/12): classical tables.
    assert S.STAG4 == [Fr(9, 8), Fr(-1, 24)]
    assert S.CENT4 == [Fr(-5, 2), Fr(4, 3), Fr(-1, 12)]


def _solve_exact(A, b):
    """Gauss-Jordan elimination over the rationals."""
    n = len(A)
    M = [list(A[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        pv = M[c][c]
        M[c] = [x / pv for x in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [M[i][n] for i in range(n)]


def test_appendix_uyy_rows_rederived():
    """Appendix A u_yy rows: the unique weights on u_0..u_8 (u_i at y = -i) exact for
    y^0 and y^2..y^9 (zero slope at the surface built in)."""
    powers = [0] + list(range(2, 10))
    for r in range(4):
        y0 = Fr(-r)
        A = [[Fr(-i) ** k for i in range(9)] for k in powers]
        b = [k * (k - 1) * y0 ** (k - 2) if k >= 2 else Fr(0) for k in powers]
        assert _solve_exact(A, b) == S.FS_UYY[r], r


def test_appendix_uy_rows_rederived():
    powers = [0] + list(range(2, 9))
    for r in range(3):
        y0 = -Fr(2 * r + 1, 2)
        A = [[Fr(-i) ** k for i in range(8)] for k in powers]
        b = [k * y0 ** (k - 1) if k >= 1 else Fr(0) for k in powers]
        assert _solve_exact(A, b) == S.FS_UY[r], r


def test_appendix_rows_not_exact_on_linear():
    """The Neumann condition is built in: y^1 is not differentiated exactly."""
    for r in range(4):
        assert sum(c * Fr(-i) for i, c in enumerate(S.FS_UYY[r])) != 0
    for r in range(3):
        assert sum(c * Fr(-i) for i, c in enumerate(S.FS_UY[r])) != 1


def test_free_surface_dwy_rows():
    """Sec. 2.2: d(w_y)/dy rows exact for w = y^k, k = 1..8 (w(0) = 0 at the surface)."""
    pts = [-Fr(2 * q + 1, 2) for q in range(8)]
    for j in range(4):
        for k in range(1, 9):
            val = sum(c * p ** k for c, p in zip(S.FS_DWY[j], pts))
            assert val == k * Fr(-j) ** (k - 1), (j, k)
        assert sum(c * p ** 9 for c, p in zip(S.FS_DWY[j], pts)) != 9 * Fr(-j) ** 8


def test_fornberg_generic_float_matches_exact():
    xs = [Fr(k) for k in (-3, -1, 0, 2, 5)]
    ex = S.fornberg_weights(Fr(1, 3), xs, 3)
    fl = S.fornberg_weights(1.0 / 3.0, [float(x) for x in xs], 3)
    for k in range(4):
        for j in range(len(xs)):
            assert abs(float(ex[k][j]) - fl[k][j]) <= 1e-12 * max(1.0, abs(float(ex[k][j])))

"""The fixed-point row sum of the constant-coefficient Laplacian (pcg_apply, default
flags) against exact rational arithmetic, and the FP64-addition row (flag
PCG_STENCIL_FP64_SUM) against its textbook error bound (GB300 only).

Exact reference: each row C*x_c - sum(neighbours) in Fractions (C*x_c exact);
float(Fraction) is the correctly rounded binary64 value.  Bound for the fixed-point row:
|y - exact| <= 0.5 ulp(y) + 6 * 2^-6 * ulp(largest term), for normal and subnormal
results alike; a row whose exact value rounds past the largest binary64 number is an
infinity.  Bound for FP64 left-to-right summation of k terms: (k - 1) * eps * sum |terms|
(plus one rounding).
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available()
    from paper_1706_05988_gb300 import build
    build.build()
    import paper_1706_05988_gb300 as pkg
    return pkg


def ulp(v: float) -> float:
    return math.ulp(v)


def rows(P, x):
    """For every unknown: its exact terms C*x_c, -x_nb... as Fractions (C*x_c is not a
    binary64 number in general, so it must not be formed in floating point)."""
    C = 6 if P.is_3d else 4
    shape = (P.nz, P.ny, P.nx)
    X = x.reshape(shape)
    out = []
    for k in range(P.nz):
        for j in range(P.ny):
            for i in range(P.nx):
                t = [C * F(X[k, j, i])]
                for dk, dj, di in ((0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)):
                    kk, jj, ii = k + dk, j + dj, i + di
                    if 0 <= kk < P.nz and 0 <= jj < P.ny and 0 <= ii < P.nx:
                        t.append(-F(X[kk, jj, ii]))
                out.append(t)
    return out


def apply_gpu(B, P, x, flags=0):
    import torch
    from paper_1706_05988_gb300 import pcg as C
    with B.Solver(P, flags=flags) as s:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        assert C.pcg_apply(s.ctx, xd, yd) == C.PCG_OK
        return yd.cpu().numpy()


def inputs(kind, n, seed):
    u = S.uniform_pm1(seed, n)
    if kind == "uniform":
        return u
    if kind == "wide":           # exponents spread over 60 binades, random signs
        return np.sign(u) * 10.0 ** (60 * S.uniform01(seed + 1, n) - 30)
    if kind == "cancel":         # nearly constant: rows cancel to a few ulps of the terms
        return 1.0 + 2.0 ** -40 * u
    if kind == "zeros":
        v = u.copy()
        v[::3] = 0.0
        v[1::7] = -0.0
        return v
    if kind == "tiny":           # near the bottom of the normal range: subnormal rows
        return 1e-306 * u
    if kind == "subnormal":      # subnormal inputs and results
        return 1e-310 * u
    if kind == "huge":           # near the top of the range: some rows overflow
        return 1.7e308 * np.sign(u) * (0.5 + 0.5 * np.abs(u))
    raise ValueError(kind)


DBL_MAX = F(np.finfo(np.float64).max)
OVERFLOW = DBL_MAX + F(2) ** 970        # halfway to 2^1024: from here on, rounding gives inf


# "3d_even": two unknowns per thread in 3D, the one stencil form whose units with an
# Inf/NaN term or a row outside the normal range are evaluated with FP64 additions; the
# others evaluate every row in fixed point.
GRIDS = [("3d", lambda: S.laplacian_3d(7, 6, 5)), ("3d_odd", lambda: S.laplacian_3d(5, 4, 3)),
         ("2d", lambda: S.laplacian_2d(12, 9)), ("2d_odd", lambda: S.laplacian_2d(9, 7)),
         ("3d_even", lambda: S.laplacian_3d(8, 6, 5))]
FP64_FALLBACK = {"3d_even"}


@pytest.mark.parametrize("gname,maker", GRIDS, ids=[g[0] for g in GRIDS])
@pytest.mark.parametrize("kind", ["uniform", "wide", "cancel", "zeros", "tiny", "subnormal", "huge"])
def test_fixed_point_rows_vs_exact(B, gname, maker, kind):
    P = maker()
    x = inputs(kind, P.n, 5)
    y = apply_gpu(B, P, x)
    # the FP64-addition rows, which the fallback of that one stencil form reproduces bit for bit
    ref = apply_gpu(B, P, x, flags=B.PCG_STENCIL_FP64_SUM) if gname in FP64_FALLBACK else None
    exact_hits = overflows = 0
    for c, terms in enumerate(rows(P, x)):
        ex = sum(terms, F(0))
        if ref is not None and (y[c] == ref[c] or (np.isnan(y[c]) and np.isnan(ref[c]))) and \
                (abs(ex) >= OVERFLOW or not np.isfinite(y[c]) or 0 < abs(ex) < 4 * F(2) ** -1022):
            continue                           # a fallback unit (only where the fast form stops)
        if abs(ex) >= OVERFLOW:
            assert y[c] == (np.inf if ex > 0 else -np.inf), (c, y[c])
            overflows += 1
            continue
        rounded = float(ex)
        big = max(abs(t) for t in terms)
        ulp_big = F(ulp(float(big))) if big <= DBL_MAX else F(2) ** 975
        bound = F(0.5 * ulp(rounded)) + F(6) * F(2) ** -6 * (ulp_big if big > 0 else F(0))
        if ref is not None and kind in ("tiny", "subnormal", "huge") and y[c] == ref[c]:
            # the other row of a fallback unit: FP64 additions, within their textbook bound
            bound = F(6 * 2.0 ** -53 * 1.01) * sum((abs(t) for t in terms), F(0)) + F(0.5 * ulp(rounded))
        assert np.isfinite(y[c]) and abs(F(y[c]) - ex) <= bound, (c, y[c], rounded, terms)
        exact_hits += y[c] == rounded
    if kind in ("uniform", "zeros") or (kind == "subnormal" and gname not in FP64_FALLBACK):
        assert exact_hits >= 0.99 * P.n        # well-scaled rows are (almost all) correctly rounded
    if kind == "huge" and gname not in FP64_FALLBACK:
        assert overflows > 0


@pytest.mark.parametrize("gname,maker", GRIDS[:3], ids=[g[0] for g in GRIDS[:3]])
def test_fp64_sum_rows_within_bound(B, gname, maker):
    P = maker()
    x = inputs("wide", P.n, 9)
    y = apply_gpu(B, P, x, flags=B.PCG_STENCIL_FP64_SUM)
    eps = 2.0 ** -53
    for c, terms in enumerate(rows(P, x)):
        ex = sum(terms, F(0))
        k = len(terms)
        bound = F((k - 1) * eps * 1.01) * sum((abs(t) for t in terms), F(0)) + F(0.5 * ulp(float(ex)))
        assert abs(F(y[c]) - ex) <= bound


@pytest.mark.parametrize("gname,maker", GRIDS, ids=[g[0] for g in GRIDS])
def test_special_values(B, gname, maker):
    """Inf and NaN inputs give what IEEE-754 addition gives in any order: NaN where a row
    meets a NaN or infinities of both signs, else the infinity (with its sign); the FP64
    addition rows agree value for value."""
    P = maker()
    x = S.uniform_pm1(3, P.n)
    x[1] = np.inf
    x[3] = -np.inf                        # row 2 sees -inf and +inf terms: NaN
    x[P.n // 2] = np.nan
    x[P.n - 2] = -np.inf
    y = apply_gpu(B, P, x)
    ref = apply_gpu(B, P, x, flags=B.PCG_STENCIL_FP64_SUM)
    assert np.isnan(y[2])
    assert np.array_equal(np.isnan(y), np.isnan(ref))
    inf = np.isinf(ref)
    assert np.array_equal(np.isinf(y), inf) and np.array_equal(y[inf], ref[inf])
    fin = np.isfinite(ref)
    np.testing.assert_allclose(y[fin], ref[fin], rtol=1e-14, atol=1e-15)


def test_order_independent(B):
    """The fixed-point row does not depend on the order of its terms: mirroring the grid
    mirrors the result bit for bit (FP64 left-to-right sums in general do not)."""
    P = S.laplacian_3d(8, 6, 4)
    x = inputs("wide", P.n, 13)
    y = apply_gpu(B, P, x).reshape(4, 6, 8)
    xm = x.reshape(4, 6, 8)[::-1, ::-1, ::-1].copy().ravel()
    ym = apply_gpu(B, P, xm).reshape(4, 6, 8)[::-1, ::-1, ::-1]
    assert np.array_equal(y, ym)

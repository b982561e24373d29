"""The fixed-point row sum of the constant-coefficient Laplacian (pcg_apply, default
flags) against exact rational arithmetic, and the FP64-addition row (flag
PCG_STENCIL_FP64_SUM) against its textbook error bound (GB300 only).

Exact reference: each row C*x_c - sum(neighbours) in Fractions (C*x_c exact);
float(Fraction) is the correctly rounded binary64 value.  Bound for the fixed-point row:
|y - exact| <= 0.5 ulp(y) + 6 * 2^-6 * ulp(largest term).  Bound for FP64
left-to-right summation of k terms: (k - 1) * eps * sum |terms| (plus one rounding).
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
    if kind == "tiny":           # near the bottom of the normal range: some rows fall back
        return 1e-306 * u
    raise ValueError(kind)


GRIDS = [("3d", lambda: S.laplacian_3d(7, 6, 5)), ("3d_odd", lambda: S.laplacian_3d(5, 4, 3)),
         ("2d", lambda: S.laplacian_2d(12, 9)), ("2d_odd", lambda: S.laplacian_2d(9, 7))]


@pytest.mark.parametrize("gname,maker", GRIDS, ids=[g[0] for g in GRIDS])
@pytest.mark.parametrize("kind", ["uniform", "wide", "cancel", "zeros", "tiny"])
def test_fixed_point_rows_vs_exact(B, gname, maker, kind):
    P = maker()
    x = inputs(kind, P.n, 5)
    y = apply_gpu(B, P, x)
    exact_hits = 0
    for c, terms in enumerate(rows(P, x)):
        ex = sum(terms, F(0))
        rounded = float(ex)
        big = float(max(abs(t) for t in terms))
        bound = F(0.5 * ulp(rounded)) + F(6) * F(2) ** -6 * F(ulp(big) if big > 0 else 0.0)
        if abs(rounded) < 2.2250738585072014e-308 * 4 or big > 1e300:
            bound += F(ulp(big)) * 8           # fallback rows: FP64 additions
        assert abs(F(y[c]) - ex) <= bound, (c, y[c], rounded, terms)
        exact_hits += y[c] == rounded
    if kind in ("uniform", "zeros"):
        assert exact_hits >= 0.99 * P.n        # well-scaled rows are (almost all) correctly rounded


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


def test_special_values_fall_back(B):
    P = S.laplacian_3d(4, 4, 4)
    x = S.uniform_pm1(3, P.n)
    x[21] = np.inf
    x[42] = np.nan
    y = apply_gpu(B, P, x)
    ref = apply_gpu(B, P, x, flags=B.PCG_STENCIL_FP64_SUM)
    assert np.array_equal(np.isnan(y), np.isnan(ref)) and np.array_equal(np.isinf(y), np.isinf(ref))
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

"""Oracle: exact rational-arithmetic CG and (shifted) pipelined CG for tiny systems.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Pure-Python Fractions, dense matrices, n <= ~12.  In exact arithmetic
Algorithms 1, 2 and 3 of arXiv 1706.05988 produce the same alpha_i, beta_i
and iterates x_i (Section 3, first paragraph); these routines are the exact
reference the FP64 oracle is pinned to.
"""
from __future__ import annotations

from fractions import Fraction as F
from typing import Optional, Sequence


def _mv(A, x):
    n = len(x)
    return [sum((A[i][j] * x[j] for j in range(n)), F(0)) for i in range(n)]


def _dot(a, b):
    return sum((x * y for x, y in zip(a, b)), F(0))


def _minv(minv, v):
    return list(v) if minv is None else [m * x for m, x in zip(minv, v)]


def cg(A, b, x0=None, iters: int = 10, minv: Optional[Sequence[F]] = None):
    """Algorithm 1.  Returns (alpha[0..k-1], beta[0..k-1] with beta[0]=0, x_k, [x_0..x_k])."""
    n = len(b)
    x = [F(0)] * n if x0 is None else [F(v) for v in x0]
    Ax = _mv(A, x)
    r = [F(bi) - ai for bi, ai in zip(b, Ax)]
    u = _minv(minv, r)
    p = list(u)
    gamma = _dot(r, u)
    alphas, betas, xs = [], [F(0)], [list(x)]
    for _ in range(iters):
        if gamma == 0:
            break
        s = _mv(A, p)
        a = gamma / _dot(s, p)
        alphas.append(a)
        x = [xi + a * pi for xi, pi in zip(x, p)]
        r = [ri - a * si for ri, si in zip(r, s)]
        u = _minv(minv, r)
        g2 = _dot(r, u)
        bt = g2 / gamma
        betas.append(bt)
        p = [ui + bt * pi for ui, pi in zip(u, p)]
        gamma = g2
        xs.append(list(x))
    return alphas, betas[:len(alphas)], x, xs


def pcg_sh(A, b, x0=None, sigma=F(0), iters: int = 10, minv: Optional[Sequence[F]] = None, gap_log=None):
    """Algorithm 3 (Algorithm 2 for sigma = 0).  Same return convention as cg().
    gap_log (a list): receives, per iteration i, the largest entry magnitudes of the gaps of
    Section 3.1: f_i = (b - A x_i) - r_i, h_i = (A u_i - sigma r_i) - w_i (at the start of
    the iteration), g_i = (A p_i - sigma t_i) - s_i and j_i = A q_i - z_i (once p_i, t_i,
    s_i, q_i, z_i are formed)."""
    n = len(b)
    sigma = F(sigma)
    x = [F(0)] * n if x0 is None else [F(v) for v in x0]
    Ax = _mv(A, x)
    r = [F(bi) - ai for bi, ai in zip(b, Ax)]
    u = _minv(minv, r)
    Au = _mv(A, u)
    w = [au - sigma * ri for au, ri in zip(Au, r)]
    z = q = s = t = p = [F(0)] * n
    alphas, betas, xs = [], [], [list(x)]
    gamma_prev = alpha_prev = None
    for i in range(iters):
        gamma = _dot(r, u)
        if gamma == 0:
            break
        delta = _dot([wi + sigma * ri for wi, ri in zip(w, r)], u)
        m = _minv(minv, w)
        nn = _mv(A, m)
        if i > 0:
            bt = gamma / gamma_prev
            a = 1 / (delta / gamma - bt / alpha_prev)
        else:
            bt = F(0)
            a = gamma / delta
        alphas.append(a)
        betas.append(bt)
        z = [ni + bt * zi for ni, zi in zip(nn, z)]
        q = [mi + bt * qi for mi, qi in zip(m, q)]
        s = [wi + bt * si for wi, si in zip(w, s)]
        t = [ri + bt * ti for ri, ti in zip(r, t)]
        p = [ui + bt * pi for ui, pi in zip(u, p)]
        if gap_log is not None:
            def mx(v):
                return max((abs(e) for e in v), default=F(0))
            f_i = [bi - ai - ri for bi, ai, ri in zip(b, _mv(A, x), r)]
            h_i = [ai - sigma * ri - wi for ai, ri, wi in zip(_mv(A, u), r, w)]
            g_i = [ai - sigma * ti - si for ai, ti, si in zip(_mv(A, p), t, s)]
            j_i = [ai - zi for ai, zi in zip(_mv(A, q), z)]
            gap_log.append({"f": mx(f_i), "g": mx(g_i), "h": mx(h_i), "j": mx(j_i)})
        x = [xi + a * pi for xi, pi in zip(x, p)]
        r = [ri - (a * si + a * sigma * ti) for ri, si, ti in zip(r, s, t)]
        u = [ui - (a * qi + a * sigma * pi) for ui, qi, pi in zip(u, q, p)]
        w = [wi - a * zi for wi, zi in zip(w, z)]
        gamma_prev, alpha_prev = gamma, a
        xs.append(list(x))
    return alphas, betas, x, xs


def pcg_varsh(A, b, shifts, x0=None, iters: int = 10, minv: Optional[Sequence[F]] = None):
    """Algorithm 4 (variable shift): shifts[0] = sigma_{-1}, shifts[k + 1] = sigma_k."""
    n = len(b)
    sg = [F(v) for v in shifts]
    x = [F(0)] * n if x0 is None else [F(v) for v in x0]
    Ax = _mv(A, x)
    r = [F(bi) - ai for bi, ai in zip(b, Ax)]
    u = _minv(minv, r)
    Au = _mv(A, u)
    w = [au - sg[0] * ri for au, ri in zip(Au, r)]
    z = q = s = t = p = [F(0)] * n
    alphas, betas, xs = [], [], [list(x)]
    gamma_prev = alpha_prev = None
    for i in range(iters):
        sp, sc = sg[i], sg[i + 1]
        ds = sc - sp
        gamma = _dot(r, u)
        if gamma == 0:
            break
        delta = _dot([wi + sp * ri for wi, ri in zip(w, r)], u)
        m = _minv(minv, w)
        nn = _mv(A, m)
        if i > 0:
            bt = gamma / gamma_prev
            a = 1 / (delta / gamma - bt / alpha_prev)
        else:
            bt = F(0)
            a = gamma / delta
        alphas.append(a)
        betas.append(bt)
        t = [ri + bt * ti for ri, ti in zip(r, t)]
        p = [ui + bt * pi for ui, pi in zip(u, p)]
        s = [wi + bt * si - ds * ti for wi, si, ti in zip(w, s, t)]
        q = [mi + bt * qi - ds * pi for mi, qi, pi in zip(m, q, p)]
        z = [ni + bt * zi - ds * (si + sc * ti) for ni, zi, si, ti in zip(nn, z, s, t)]
        x = [xi + a * pi for xi, pi in zip(x, p)]
        w = [wi - a * zi - ds * ri for wi, zi, ri in zip(w, z, r)]
        r = [ri - (a * si + a * sc * ti) for ri, si, ti in zip(r, s, t)]
        u = [ui - (a * qi + a * sc * pi) for ui, qi, pi in zip(u, q, p)]
        gamma_prev, alpha_prev = gamma, a
        xs.append(list(x))
    return alphas, betas, x, xs

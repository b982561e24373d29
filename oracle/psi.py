"""Oracle: local rounding-error propagation analysis and shift selection.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 3.2 of arXiv 1706.05988:
  P_k(sigma)       the 4x4 local error propagation matrix, Eq. (propmat_shifted),
                   built from iteration k's alpha_k, beta_k;
  P_{j,i}(sigma)   = P_i P_{i-1} ... P_j, Eq. (matrix_product);
  psi_i(sigma)     = max_{1<=j<=i} ||P_{j,i}(sigma)||_2, Eq. (functionpsi);
  P_k(sigma_{k-1}, sigma_k)  the variable-shift matrix of Section 4.1, Eq. (propmat_varshifted).
Section 5.1: the shift is chosen a posteriori, minimising psi_i over sigma,
from the alpha/beta history of the unshifted pipelined CG run.

The spectral norm is numpy's (a LAPACK SVD), a library step.
"""
from __future__ import annotations

import numpy as np


def prop_matrix(alpha: float, beta: float, sigma: float) -> np.ndarray:
    """P_k(sigma) of Eq. (propmat_shifted) for scalars alpha_k, beta_k."""
    a, b, s = alpha, beta, sigma
    return np.array([[1.0, -a * b, -a, 0.0],
                     [0.0, b, 1.0, 0.0],
                     [0.0, -a * b * s, 1.0 - a * s, -a * b],
                     [0.0, 0.0, 0.0, b]])


def psi(alpha, beta, i: int, sigma: float) -> float:
    """psi_i(sigma): alpha/beta are indexed by iteration (entries 1..i are used)."""
    Q = np.eye(4)
    best = 0.0
    for j in range(i, 0, -1):                 # Q = P_i ... P_j, extended on the right
        Q = Q @ prop_matrix(alpha[j], beta[j], sigma)
        best = max(best, float(np.linalg.norm(Q, 2)))
    return best


def prop_matrix_var(alpha: float, beta: float, s_prev: float, s_cur: float) -> np.ndarray:
    """P_k(sigma_{k-1}, sigma_k) of Eq. (propmat_varshifted), Section 4.1: the variable-shift
    propagation matrix.  Its last row couples the j-gap to g and h through the change of
    shift; with s_prev == s_cur it is P_k(sigma) of Eq. (propmat_shifted)."""
    a, b, d = alpha, beta, s_cur - s_prev
    return np.array([[1.0, -a * b, -a, 0.0],
                     [0.0, b, 1.0, 0.0],
                     [0.0, -a * b * s_prev, 1.0 - a * s_prev, -a * b],
                     [0.0, -b * d, -d, b]])


def psi_varsh(alpha, beta, i: int, shifts) -> float:
    """psi_i for a shift schedule: shifts[0] = sigma_{-1}, shifts[k + 1] = sigma_k, so that
    P_j = P_j(sigma_{j-1}, sigma_j) = P(alpha_j, beta_j, shifts[j], shifts[j + 1])."""
    Q = np.eye(4)
    best = 0.0
    for j in range(i, 0, -1):
        Q = Q @ prop_matrix_var(alpha[j], beta[j], shifts[j], shifts[j + 1])
        best = max(best, float(np.linalg.norm(Q, 2)))
    return best


def psi_history(alpha, beta, sigma: float, imax: int) -> np.ndarray:
    """psi_i(sigma) for i = 1..imax (the right panel of Fig. 2)."""
    return np.array([psi(alpha, beta, i, sigma) for i in range(1, imax + 1)])


def select_sigma(alpha, beta, i: int, grid, slack: float = 2.0) -> tuple[float, np.ndarray]:
    """Shift choice from psi_i on a grid; returns (sigma*, psi values on the grid).

    psi_i(sigma) keeps falling as sigma approaches the top of the spectrum and
    then explodes (a too large shift destroys convergence, Section 5.1), so the
    raw argmin sits at the edge of that cliff.  The shifts of Table 1 lie near
    the minimum but well inside the cliff (lapl200: sigma* = 4 for a spectrum
    in (0, 8)).  Reading taken: sigma* = the smallest grid shift whose psi is
    within `slack` times the grid minimum."""
    grid = np.asarray(grid, dtype=np.float64)
    vals = np.array([psi(alpha, beta, i, s) for s in grid])
    ok = np.where(vals <= slack * np.nanmin(vals))[0]
    return float(np.min(grid[ok])), vals

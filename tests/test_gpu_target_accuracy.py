"""Attainable accuracy at the full workloads against stored oracle runs (GB300 only).

The oracle needs minutes for these runs, so tests/golden/make_full_size_golden.py (which
calls only oracle/ and synthetic/) ran them once and stored what is compared here:

* 256^3 7-point Laplacian, shifted p-CG (Algorithm 3) with sigma = 6, 1,000 iterations, as a
  matrix-free stencil and as CSR int32 -- the benchmark's solve.  The final true relative
  residual ||b - A x|| / ||b|| must lie within a factor 10 of the oracle's (the accuracy half of
  the performance target), the recursive residual must follow the oracle's path, and alpha_i,
  beta_i the oracle's.
* 128^3 FV diffusion with kappa = 10^U[-3,3] on 8^3 blocks, Jacobi M^-1, sigma = 0.75, to
  ||r_i|| <= 1e-10 ||b||: iterations, final true residual and the iterate at 4,096 seeded
  indices, in binary64 and in mixed precision with binary64 refinement.
"""
import json
import os

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL_SCALARS = 1e-10


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1706_05988_gb300 import build
    build.build()
    import paper_1706_05988_gb300 as pkg
    return pkg


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


@pytest.fixture(scope="module")
def lapl256():
    P, b, _ = S.poisson3d_manufactured(256)
    return P, b


@pytest.mark.parametrize("form", ["stencil", "csr"])
def test_256cubed_1000_iterations_vs_oracle(B, lapl256, form):
    P, b = lapl256
    G = golden("spcg_256cubed_1000it.json" if form == "stencil" else "spcg_256cubed_csr_1000it.json")
    if form == "csr":
        P = S.to_csr(P)
    assert G["n"] == P.n and G["iters"] == 1000
    with B.Solver(P) as s:
        g = s.solve(b, method="spcg", sigma=6.0, maxit=1000, true_every=0)
    assert g.iters == 1000
    bn = np.linalg.norm(b)
    assert abs(bn - G["bnorm"]) <= 1e-14 * bn
    # the target's accuracy half: final true relative residual within 10x of the oracle's
    ot = G["final_true_relres"]
    assert 0.1 * ot <= g.final_true_relres <= 10 * ot, (g.final_true_relres, ot)
    # the recursive residual follows the oracle's path: to 1e-6 over the first 200
    # iterations, then within 2x (rounding differences grow with the iteration count)
    idx = np.array(G["rec_path"]["index"])
    orec = np.array(G["rec_path"]["rec_relres"])
    grec = g.rec[idx] / bn
    early = idx <= 200
    assert np.all(rel(grec[early], orec[early]) <= 1e-6), rel(grec[early], orec[early]).max()
    assert np.all((grec > 0.5 * orec) & (grec < 2.0 * orec))
    # alpha_i, beta_i: the first 20 at the parity bar, every 50th to 1e-6
    si = np.array(G["scalars"]["index"])
    oa, ob = np.array(G["scalars"]["alpha"]), np.array(G["scalars"]["beta"])
    first = si < 20
    assert np.all(rel(g.alpha[si[first]], oa[first]) <= TOL_SCALARS)
    assert np.all(rel(g.beta[si[first]][1:], ob[first][1:]) <= TOL_SCALARS)
    assert np.all(rel(g.alpha[si], oa) <= 1e-6), rel(g.alpha[si], oa).max()
    assert np.all(rel(g.beta[si][1:], ob[1:]) <= 1e-6)


@pytest.fixture(scope="module")
def varcoef128():
    P = S.varcoef_3d(128, block=8, seed=0)
    b = S.normal(1, P.n)
    return P, b, golden("varcoef128_jacobi_spcg_1e-10.json")


def test_varcoef128_fp64_jacobi_vs_oracle(B, varcoef128):
    """Binary64 with Jacobi to 1e-10: the same iteration count (to 2 %), a final true residual
    within 10x of the oracle's, and the iterate itself: the two runs differ only in rounding,
    and x agrees at the sampled indices to 1e-6 relative (in norm) although kappa ~ 1e7."""
    P, b, G = varcoef128
    with B.Solver(P, flags=B.PCG_JACOBI) as s:
        g = s.solve(b, method="spcg", sigma=0.75, tol=1e-10, maxit=40000)
    assert g.status == B.PCG_OK and G["status"] == 1
    assert abs(g.iters - G["iters"]) <= 0.02 * G["iters"] + 2, (g.iters, G["iters"])
    ot = G["final_true_relres"]
    assert 0.1 * ot <= g.final_true_relres <= 10 * ot, (g.final_true_relres, ot)
    idx = np.array(G["x_sample"]["index"])
    ox = np.array(G["x_sample"]["value"])
    err = np.linalg.norm(g.x[idx] - ox) / np.linalg.norm(ox)
    assert err <= 1e-6, err
    assert abs(np.linalg.norm(g.x) - G["x_norm"]) <= 1e-6 * G["x_norm"]


def test_varcoef128_mixed_jacobi_vs_oracle(B, varcoef128):
    """Mixed precision (binary32 auxiliary vectors, binary64 x, r, dots and refinement) with
    Jacobi to a true relative residual of 1e-10.  Its error against the oracle's converged x is
    bounded by the residual: ||x - x_o|| / ||x_o|| <= 2e-10 kappa ~ 2e-3 for kappa ~ 1e7; the
    sampled entries must meet that bound."""
    P, b, G = varcoef128
    with B.Solver(P, flags=B.PCG_JACOBI) as s:
        g = s.solve(b, method="spcg", sigma=0.75, tol=1e-10, maxit=40000, precision=B.PCG_MIXED_IR)
    assert g.status == B.PCG_OK
    assert g.final_true_relres <= 1e-10
    idx = np.array(G["x_sample"]["index"])
    ox = np.array(G["x_sample"]["value"])
    err = np.linalg.norm(g.x[idx] - ox) / np.linalg.norm(ox)
    assert err <= 2e-3, err
    assert abs(np.linalg.norm(g.x) - G["x_norm"]) <= 2e-3 * G["x_norm"]

"""Mixed precision with iterative refinement (precision PCG_MIXED_IR), GB300 only.

The paper fixes no result for this variant; what is checked is that the binary64
true residual, recomputed independently by the oracle's operator on the CPU,
reaches the requested tolerance, that the early scalars follow the FP64 oracle
to binary32 accuracy, and that every restart lowers the true residual.
"""
import numpy as np
import pytest

import oracle
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


def true_relres(P, b, x):
    return np.linalg.norm(b - oracle.apply(P, x)) / np.linalg.norm(b)


CASES = [("poisson2d_100", lambda: S.poisson2d_manufactured(100)[:2], 4.0),
         ("lapl3d_48", lambda: S.poisson3d_manufactured(48)[:2], 6.0),
         ("lapl3d_odd", lambda: (S.laplacian_3d(33, 30, 17), S.normal(2, 33 * 30 * 17)), 6.0),
         ("csr_lapl3d", lambda: (S.to_csr(S.laplacian_3d(24)), S.normal(3, 24 ** 3)), 6.0)]


@pytest.mark.parametrize("name,maker,sigma", CASES, ids=[c[0] for c in CASES])
def test_mixed_ir_reaches_tolerance(B, name, maker, sigma):
    from paper_1706_05988_gb300 import pcg as C
    P, b = maker()
    with B.Solver(P) as s:
        r = s.solve(b, method="spcg", sigma=sigma, tol=1e-10, maxit=20000, precision=C.PCG_MIXED_IR)
    assert r.status == B.PCG_OK, C.STATUS_NAMES[r.status]
    tr = true_relres(P, b, r.x)
    assert tr <= 1e-10 and abs(tr - r.final_true_relres) <= 1e-3 * tr + 1e-16
    # the refinement: the true residual at consecutive restarts decreases
    t = r.true[~np.isnan(r.true)]
    assert len(t) >= 2 and np.all(np.diff(t[:-1]) < 0)
    # against the FP64 oracle's solution
    o = oracle.pcg_sh(P, b, sigma=sigma, maxit=5000, rtol=1e-12, log_every=0)
    assert np.linalg.norm(r.x - o.x) <= 1e-6 * np.linalg.norm(o.x)


def test_mixed_first_scalars_follow_fp64(B):
    """Before the first restart the mixed iteration is Algorithm 3 with binary32 auxiliary
    vectors: alpha_i, beta_i agree with the FP64 oracle to binary32 accuracy."""
    from paper_1706_05988_gb300 import pcg as C
    P, b, _ = S.poisson3d_manufactured(40)
    with B.Solver(P) as s:
        C.pcg_set_param(s.ctx, C.PCG_PARAM_MIXED_ETA, 1e-6)
        r = s.solve(b, method="spcg", sigma=6.0, maxit=20, precision=C.PCG_MIXED_IR)
    o = oracle.pcg_sh(P, b, sigma=6.0, maxit=20, log_every=0)
    assert r.iters == 20
    np.testing.assert_allclose(r.alpha, o.alpha, rtol=1e-5)
    np.testing.assert_allclose(r.beta[1:], o.beta[1:], rtol=1e-5)


def test_mixed_stall_is_reported(B):
    """High-contrast coefficients (10^U[-3,3] blocks) without a preconditioner: the binary32
    inner solves cannot lower the true residual and the solve stops as not converged."""
    from paper_1706_05988_gb300 import pcg as C
    P = S.varcoef_3d(32, block=8, seed=0)
    b = S.normal(0, P.n)
    with B.Solver(P) as s:
        r = s.solve(b, method="spcg", sigma=0.5 * float(np.median(P.diag)), tol=1e-10, maxit=20000,
                    precision=C.PCG_MIXED_IR)
        msg = C.pcg_last_error(s.ctx)
    if r.status == B.PCG_OK:            # converged after all: the result must be right
        assert true_relres(P, b, r.x) <= 1e-10
    else:
        assert r.status == B.PCG_ENOTCONV and ("stalled" in msg or r.iters == 20000)


def test_mixed_parameters(B):
    from paper_1706_05988_gb300 import pcg as C
    P, b, _ = S.poisson2d_manufactured(16)
    with B.Solver(P) as s:
        assert C.pcg_set_param(s.ctx, C.PCG_PARAM_MIXED_ETA, 0.0) == C.PCG_EINVAL
        assert C.pcg_set_param(s.ctx, C.PCG_PARAM_MIXED_ETA, 1.5) == C.PCG_EINVAL
        assert C.pcg_set_param(s.ctx, C.PCG_PARAM_MAX_RESTARTS, 0) == C.PCG_EINVAL
        assert C.pcg_set_param(s.ctx, 99, 1.0) == C.PCG_EINVAL
        assert C.pcg_set_param(s.ctx, C.PCG_PARAM_MAX_RESTARTS, 1) == C.PCG_OK
        r = s.solve(b, method="spcg", sigma=2.0, tol=1e-14, maxit=5000, precision=C.PCG_MIXED_IR)
        assert r.status == B.PCG_ENOTCONV      # one restart allowed: stops after it


# ------------------------------------------------------------------ with the Jacobi preconditioner

def diag_of(P):
    if P.layout == S.CSR32:
        d = np.zeros(P.n)
        rows = np.repeat(np.arange(P.n), np.diff(P.row_ptr))
        np.add.at(d, rows[P.col == rows], P.val[P.col == rows])
        return d
    if P.constant:
        return np.full(P.n, 6.0 if P.is_3d else 4.0)
    return np.asarray(P.diag, dtype=np.float64)


JAC_CASES = [("varcoef3d_32_k1e6", lambda: S.varcoef_3d(32, block=8, seed=0), 1.0),
             ("varcoef2d_77x53", lambda: S.varcoef_2d(77, 53, seed=2), 1.0),
             ("lapl3d_odd", lambda: S.laplacian_3d(33, 30, 17), 1.0),
             ("csr_sdd", lambda: S.random_sdd_csr(20011, seed=4), 1.0)]


@pytest.mark.parametrize("name,maker,sigma", JAC_CASES, ids=[c[0] for c in JAC_CASES])
def test_mixed_jacobi_reaches_tolerance(B, name, maker, sigma):
    """Jacobi-preconditioned mixed precision reaches 1e-10 on the high-contrast coefficients that
    stall the unpreconditioned inner solves; the true residual is recomputed by the oracle's operator."""
    from paper_1706_05988_gb300 import pcg as C
    P = maker()
    b = S.normal(5, P.n)
    with B.Solver(P, flags=B.PCG_JACOBI) as s:
        r = s.solve(b, method="spcg", sigma=sigma, tol=1e-10, maxit=20000, precision=C.PCG_MIXED_IR)
    assert r.status == B.PCG_OK, C.STATUS_NAMES[r.status]
    tr = true_relres(P, b, r.x)
    assert tr <= 1e-10 and abs(tr - r.final_true_relres) <= 1e-3 * tr + 1e-16
    t = r.true[~np.isnan(r.true)]
    assert len(t) >= 2 and np.all(np.diff(t[:-1]) < 0)
    # the FP64 oracle with the same M^-1 reaches the same solution (to what kappa allows at 1e-10)
    o = oracle.pcg_sh(P, b, sigma=sigma, maxit=20000, rtol=1e-12, minv=1.0 / diag_of(P), log_every=0)
    assert o.status == 1
    assert np.linalg.norm(r.x - o.x) <= 1e-3 * np.linalg.norm(o.x)


def test_mixed_jacobi_first_scalars_follow_fp64(B):
    """Before the first restart: Algorithm 3 with M^-1 = D^-1 and binary32 auxiliary vectors."""
    from paper_1706_05988_gb300 import pcg as C
    P = S.varcoef_3d(24, block=4, seed=1)
    b = S.normal(6, P.n)
    with B.Solver(P, flags=B.PCG_JACOBI) as s:
        C.pcg_set_param(s.ctx, C.PCG_PARAM_MIXED_ETA, 1e-6)
        r = s.solve(b, method="spcg", sigma=1.0, maxit=20, precision=C.PCG_MIXED_IR)
    o = oracle.pcg_sh(P, b, sigma=1.0, maxit=20, minv=1.0 / diag_of(P), log_every=0)
    assert r.iters == 20
    np.testing.assert_allclose(r.alpha, o.alpha, rtol=1e-4)
    np.testing.assert_allclose(r.beta[1:], o.beta[1:], rtol=1e-4)


def test_mixed_variable_shift_not_implemented(B):
    from paper_1706_05988_gb300 import pcg as C
    P = S.laplacian_2d(16)
    with B.Solver(P, flags=B.PCG_JACOBI) as s:
        assert B.pcg_set_shifts(s.ctx, np.linspace(1.0, 0.5, 11)) == B.PCG_OK
        r = s.solve(np.ones(P.n), method="spcg", maxit=10, precision=C.PCG_MIXED_IR, raise_on_error=False)
        assert r.status == B.PCG_ENOTIMPL

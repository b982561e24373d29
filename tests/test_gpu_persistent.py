"""Persistent cooperative form of the iteration (flag PCG_PERSISTENT), GB300 only:
parity with the oracle, agreement with the launch-per-iteration form, and the
bounded grid-barrier wait (a barrier that waits for arrivals that never come ends
with PCG_ETIMEOUT and leaves the context usable)."""
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


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(np.abs(np.asarray(b)), 1e-300))


SHAPES = [("poisson2d_100", lambda: S.poisson2d_manufactured(100)[:2], 4.0),
          ("lapl3d_odd", lambda: (S.laplacian_3d(21, 17, 13), S.normal(1, 21 * 17 * 13)), 6.0),
          ("lapl3d_64", lambda: S.poisson3d_manufactured(64)[:2], 6.0),
          ("var2d", lambda: (S.varcoef_2d(64, 48, seed=2), S.normal(2, 64 * 48)), 1.0),
          ("csr", lambda: (S.to_csr(S.laplacian_3d(20)), S.normal(3, 8000)), 6.0)]


@pytest.mark.parametrize("name,maker,sigma", SHAPES, ids=[s[0] for s in SHAPES])
def test_persistent_vs_oracle(B, name, maker, sigma):
    P, b = maker()
    with B.Solver(P, flags=B.PCG_PERSISTENT) as s:
        g = s.solve(b, method="spcg", sigma=sigma, maxit=20)
    o = oracle.pcg_sh(P, b, sigma=sigma, maxit=20, log_every=20)
    assert g.iters == o.iters == 20
    assert rel(g.alpha, o.alpha) <= 1e-10 and rel(g.beta[1:], o.beta[1:]) <= 1e-10
    assert np.linalg.norm(g.x - o.x) <= 1e-8 * np.linalg.norm(o.x)
    bn = np.linalg.norm(b)
    assert 0.1 <= g.final_true_relres / (o.true[-1] / bn) <= 10


def test_persistent_matches_launch_per_iteration(B):
    P, b, _ = S.poisson3d_manufactured(48)
    with B.Solver(P, flags=B.PCG_PERSISTENT) as sp, B.Solver(P) as sl:
        a = sp.solve(b, method="spcg", sigma=6.0, tol=1e-10, maxit=2000)
        a2 = sp.solve(b, method="spcg", sigma=6.0, tol=1e-10, maxit=2000)
        l = sl.solve(b, method="spcg", sigma=6.0, tol=1e-10, maxit=2000)
    assert a.status == l.status == B.PCG_OK
    assert abs(a.iters - l.iters) <= 1
    k = min(a.iters, l.iters)
    assert rel(a.rec[:k], l.rec[:k]) < 1e-6
    assert np.array_equal(a.x, a2.x)                      # deterministic
    assert a.final_true_relres <= 1.5e-10


def test_persistent_breakdown_and_pcg(B):
    n = 64
    d = np.ones(n)
    d[::2] = -1.0
    P = S.Problem(S.CSR32, row_ptr=np.arange(n + 1, dtype=np.int32), col=np.arange(n, dtype=np.int32), val=d,
                  n_csr=n)
    with B.Solver(P, flags=B.PCG_PERSISTENT) as s:
        r = s.solve(np.ones(n), method="spcg", sigma=0.5, maxit=10)
    assert r.status == B.PCG_EBREAKDOWN
    P2, b2, _ = S.poisson2d_manufactured(40)
    with B.Solver(P2, flags=B.PCG_PERSISTENT) as s:
        p = s.solve(b2, method="pcg", maxit=30)
    o = oracle.pcg_sh(P2, b2, sigma=0.0, maxit=30, log_every=0)
    assert rel(p.alpha, o.alpha) <= 1e-10


def test_barrier_wait_times_out_and_context_recovers(B):
    from paper_1706_05988_gb300 import pcg as C
    P, b, _ = S.poisson3d_manufactured(32)
    with B.Solver(P, flags=B.PCG_PERSISTENT) as s:
        assert C.pcg_set_param(s.ctx, C.PCG_PARAM_BARRIER_TIMEOUT_MS, 50) == C.PCG_OK
        assert C.pcg_set_param(s.ctx, C.PCG_PARAM_TEST_BARRIER_PHANTOMS, 1) == C.PCG_OK
        r = s.solve(b, method="spcg", sigma=6.0, maxit=100, raise_on_error=False)
        assert r.status == C.PCG_ETIMEOUT
        assert "time limit" in C.pcg_last_error(s.ctx)
        assert C.pcg_set_param(s.ctx, C.PCG_PARAM_TEST_BARRIER_PHANTOMS, 0) == C.PCG_OK
        ok = s.solve(b, method="spcg", sigma=6.0, maxit=100)
    o = oracle.pcg_sh(P, b, sigma=6.0, maxit=100, log_every=0)
    assert ok.iters == 100 and np.linalg.norm(ok.x - o.x) <= 1e-8 * np.linalg.norm(o.x)

"""The per-cluster solvers of the batched launch and of the server against the oracle,
iteration by iteration (GB300 only).

Each cluster runs its own copy of Algorithm 3's recurrences and a DSMEM cluster reduction,
so the solvers record alpha_i, beta_i of their first iterations (pcg_batch_scalars;
pcg_poll's alpha_hist/beta_hist).  These are compared with the oracle's:
* binary64, M = I and Jacobi: 1e-10 relative over 20 iterations (the parity bar of the
  single-system kernels), for every operator family, one system in each size class of the
  batch (n < 8,192; < 65,536; larger), and both register variants of the batch kernel;
  and every entry of x after 15 iterations;
* mixed precision (binary32 auxiliary vectors): 1e-5 relative over the iterations before
  the first restart (binary32 rounding of the vectors moves the scalars by ~1e-7 per
  iteration, amplified by the Krylov process).
"""
import numpy as np
import pytest

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5
K = 20


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available()
    from paper_1706_05988_gb300 import build
    build.build()
    import paper_1706_05988_gb300 as pkg
    return pkg


def diag_of(P):
    c = S.to_csr(P)
    rows = np.repeat(np.arange(c.n), np.diff(c.row_ptr))
    d = np.zeros(c.n)
    np.add.at(d, rows[c.col == rows], c.val[c.col == rows])
    return d


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


# one family per batch; a system in each size class (the last one has n >= 65,536)
FAMILIES = {
    "lapl2d": lambda: [S.laplacian_2d(50, 40), S.laplacian_2d(150, 130), S.laplacian_2d(300, 260)],
    "var2d": lambda: [S.varcoef_2d(40, 40, seed=1), S.varcoef_2d(120, 120, seed=2), S.varcoef_2d(300, 300, seed=3)],
    "lapl3d": lambda: [S.laplacian_3d(16, 15, 14), S.laplacian_3d(30, 28, 26), S.laplacian_3d(48)],
    "var3d": lambda: [S.varcoef_3d(16, block=4, seed=4), S.varcoef_3d(32, block=8, seed=5),
                      S.varcoef_3d(44, block=4, seed=6)],
    "csr": lambda: [S.to_csr(S.laplacian_3d(12, 11, 10)), S.random_sdd_csr(20000, seed=7),
                    S.to_csr(S.varcoef_3d(42, block=6, seed=8))],
}


def shift_of(P, jacobi):
    return 1.0 if jacobi else 0.5 * float(np.median(diag_of(P)))


def live_count(o, k):
    """Iterations whose scalars are compared: while ||r_i|| > 1e-9 ||r_0|| (past that the
    scalars carry rounding noise of the converged solve on both sides)."""
    return int(min(k, np.sum(o.rec[:k] > 1e-9 * o.rec[0])))


@pytest.mark.parametrize("jacobi", [False, True], ids=["m_identity", "jacobi"])
@pytest.mark.parametrize("occ", [2, 4])
@pytest.mark.parametrize("fam", list(FAMILIES))
def test_batch_fp64_scalars_vs_oracle(B, fam, occ, jacobi):
    probs = FAMILIES[fam]()
    assert probs[-1].n >= 65536 and probs[0].n < 8192 and 8192 <= probs[1].n < 65536
    bs = [S.normal(300 + i, P.n) for i, P in enumerate(probs)]
    sig = [shift_of(P, jacobi) for P in probs]
    with B.Batch(probs, flags=B.PCG_JACOBI if jacobi else 0) as bt:
        for c in range(3):
            assert bt.set_class_occupancy(c, occ) == B.PCG_OK
        xs, it, st, tr = bt.solve(bs, sig, tol=0.0, maxit=K)
        al, be = bt.scalars(K)
    for i, (P, b, s) in enumerate(zip(probs, bs, sig)):
        minv = 1.0 / diag_of(P) if jacobi else None
        o = oracle.pcg_sh(P, b, sigma=s, maxit=K, log_every=0, minv=minv)
        assert it[i] == o.iters == K
        k = live_count(o, K)
        assert np.all(rel(al[i, :k], o.alpha[:k]) <= TOL64), (i, rel(al[i, :k], o.alpha[:k]).max())
        assert be[i, 0] == 0.0 and np.all(rel(be[i, 1:k], o.beta[1:k]) <= TOL64)


@pytest.mark.parametrize("fam", list(FAMILIES))
def test_batch_iterate_after_15_iterations(B, fam):
    """Every entry of x_15 of every system against the oracle's."""
    probs = FAMILIES[fam]()
    bs = [S.normal(400 + i, P.n) for i, P in enumerate(probs)]
    sig = [shift_of(P, False) for P in probs]
    with B.Batch(probs) as bt:
        xs, it, st, tr = bt.solve(bs, sig, tol=0.0, maxit=15)
    for P, b, s, x in zip(probs, bs, sig, xs):
        o = oracle.pcg_sh(P, b, sigma=s, maxit=15, log_every=0)
        scale = np.abs(o.x).max()
        assert np.all(np.abs(x - o.x) <= 1e-10 * np.abs(o.x) + 1e-12 * scale)


def first_restart(be):
    """Index of the first restart in a mixed-precision log (beta = 0 again after i = 0)."""
    z = np.nonzero(be[1:] == 0.0)[0]
    return int(z[0]) + 1 if z.size else len(be)


@pytest.mark.parametrize("fam,jacobi", [("lapl2d", False), ("lapl3d", False), ("var2d", True), ("var3d", True),
                                        ("csr", True), ("lapl3d", True)])
def test_batch_mixed_scalars_vs_oracle(B, fam, jacobi):
    """Mixed precision: binary32 level until the first restart (large systems take the wide
    binary32 sweeps).  Only the scalars are compared here; convergence of the mixed forms is
    tested in test_gpu_batch.py."""
    probs = FAMILIES[fam]()
    bs = [S.normal(500 + i, P.n) for i, P in enumerate(probs)]
    sig = [shift_of(P, jacobi) for P in probs]
    with B.Batch(probs, flags=B.PCG_JACOBI if jacobi else 0, precision=B.PCG_MIXED_IR) as bt:
        xs, it, st, tr = bt.solve(bs, sig, tol=1e-8, maxit=20000)
        al, be = bt.scalars(K)
    for i, (P, b, s) in enumerate(zip(probs, bs, sig)):
        minv = 1.0 / diag_of(P) if jacobi else None
        o = oracle.pcg_sh(P, b, sigma=s, maxit=K, log_every=0, minv=minv)
        k = min(first_restart(be[i]), live_count(o, K), 12)
        assert k >= 8, (i, k)
        assert np.all(rel(al[i, :k], o.alpha[:k]) <= TOL32), (i, rel(al[i, :k], o.alpha[:k]).max())
        assert np.all(rel(be[i, 1:k], o.beta[1:k]) <= TOL32)


SERVED = [("lapl2d_small", lambda: S.laplacian_2d(60, 50), 0, "fp64"),
          ("var2d_large_lane", lambda: S.varcoef_2d(300, 300, seed=3), 0, "fp64"),
          ("csr_small", lambda: S.random_sdd_csr(5000, seed=9), 0, "fp64"),
          ("var3d_jacobi", lambda: S.varcoef_3d(36, block=6, seed=10), 1, "fp64"),
          ("lapl3d_mixed", lambda: S.laplacian_3d(40), 0, "mixed"),
          ("csr_mixed_jacobi", lambda: S.to_csr(S.varcoef_3d(42, block=6, seed=8)), 1, "mixed"),
          ("lapl3d_device_lane", lambda: S.laplacian_3d(84), 0, "fp64")]


def test_served_scalars_vs_oracle(B):
    """Requests of every lane (small and large cluster lanes, and n >= 2^19 on the device
    lane) submitted together; each poll returns the request's first alpha_i, beta_i."""
    from paper_1706_05988_gb300 import pcg as C
    reqs = []
    with B.Server(8 << 30, 32) as srv:
        for name, maker, jac, prec in SERVED:
            P = maker()
            b = S.normal(600 + len(reqs), P.n)
            s = shift_of(P, jac == 1)
            t = srv.submit(P, b, tol=1e-8, method=C.PCG_SPCG, sigma=s, maxit=20000,
                           flags=C.PCG_JACOBI if jac else 0,
                           precision=C.PCG_MIXED_IR if prec == "mixed" else C.PCG_FP64)
            reqs.append((name, P, b, s, jac, prec, t))
        done = {}
        import time
        t0 = time.time()
        while len(done) < len(reqs) and time.time() - t0 < 120:
            for name, P, b, s, jac, prec, t in reqs:
                if name in done:
                    continue
                r = srv.poll(t, scalars=True)
                if r is not None:
                    done[name] = r
        assert len(done) == len(reqs)
    for name, P, b, s, jac, prec, t in reqs:
        code, x, iters, trr, al, be = done[name]
        assert code == C.PCG_OK and trr <= 1.01e-8, (name, code, trr)
        minv = 1.0 / diag_of(P) if jac else None
        o = oracle.pcg_sh(P, b, sigma=s, maxit=K, log_every=0, minv=minv)
        if prec == "fp64":
            k = live_count(o, min(K, len(al)))
            tol = TOL64
        else:
            k = min(first_restart(be), live_count(o, K), 12)
            tol = TOL32
        assert k >= 8, (name, k)
        assert np.all(rel(al[:k], o.alpha[:k]) <= tol), (name, rel(al[:k], o.alpha[:k]).max())
        assert be[0] == 0.0 and np.all(rel(be[1:k], o.beta[1:k]) <= tol), name

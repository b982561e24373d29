"""Batched persistent launch (pcg_batch_*), GB300 only: every system of a batch gets
the same result as the single-system solver, for every cluster shape."""
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


def shift(P):
    c = S.to_csr(P)
    rows = np.repeat(np.arange(c.n), np.diff(c.row_ptr))
    return 0.5 * float(np.median(c.val[c.col == rows]))


def var2d_batch(k=10, seed=0):
    rng = np.random.default_rng(seed)
    sides = rng.integers(8, 80, size=(k, 2))
    probs = [S.varcoef_2d(int(a), int(b), seed=seed + i) for i, (a, b) in enumerate(sides)]
    bs = [S.normal(100 + i, P.n) for i, P in enumerate(probs)]
    return probs, bs


@pytest.mark.parametrize("cluster", [1, 2, 4, 8, 16])
def test_batch_matches_single_solver(B, cluster):
    probs, bs = var2d_batch()
    sig = [shift(P) for P in probs]
    with B.Batch(probs) as bt:
        assert bt.set_cluster(cluster) == B.PCG_OK
        xs, it, st, tr = bt.solve(bs, sig, tol=1e-9, maxit=5000)
    for P, b, s, x, i, code, t in zip(probs, bs, sig, xs, it, st, tr):
        with B.Solver(P) as one:
            r = one.solve(b, method="spcg", sigma=s, tol=1e-9, maxit=5000)
        assert code == B.PCG_OK and r.status == B.PCG_OK
        # the reduction order differs (per-block partials of a cluster vs of the whole grid), and
        # these high-contrast systems take ~10^3 iterations: the stop may move by a few iterations
        assert abs(int(i) - r.iters) <= 0.02 * r.iters + 2
        tt = np.linalg.norm(b - oracle.apply(P, x)) / np.linalg.norm(b)
        assert tt <= 3e-9 and abs(t - tt) <= 1e-6 * tt + 1e-15
        # both iterates solve the system to the tolerance: their difference is bounded by it
        assert np.linalg.norm(x - r.x) <= 1e-4 * np.linalg.norm(r.x)


def test_batch_first_iterations_vs_oracle(B):
    probs = [S.laplacian_3d(12, 10, 9), S.laplacian_3d(17, 5, 20), S.laplacian_3d(4, 4, 4)]
    bs = [S.normal(7 + i, P.n) for i, P in enumerate(probs)]
    with B.Batch(probs) as bt:
        xs, it, st, tr = bt.solve(bs, [6.0] * 3, tol=0.0, maxit=15)
    for P, b, x, i in zip(probs, bs, xs, it):
        o = oracle.pcg_sh(P, b, sigma=6.0, maxit=15, log_every=0)
        assert i == o.iters == 15 or (o.status == 1 and i == o.iters)
        assert np.linalg.norm(x - o.x) <= 1e-9 * np.linalg.norm(o.x)


def test_batch_csr_and_autotune(B):
    probs = [S.to_csr(S.laplacian_3d(n)) for n in (6, 9, 14, 20, 11)]
    bs = [S.normal(i, P.n) for i, P in enumerate(probs)]
    with B.Batch(probs) as bt:
        c, ms = bt.autotune(bs, [6.0] * 5, probe_iters=20)
        assert c in (1, 2, 4, 8, 16) and np.isfinite(ms).any()
        xs, it, st, tr = bt.solve(bs, [6.0] * 5, tol=1e-10, maxit=3000)
    assert np.all(st == B.PCG_OK) and np.all(tr <= 2e-10)
    for P, b, x in zip(probs, bs, xs):
        assert np.linalg.norm(b - oracle.apply(P, x)) <= 2e-10 * np.linalg.norm(b)


def test_batch_rejects_mixed_families(B):
    from paper_1706_05988_gb300 import pcg as C
    with pytest.raises(C.PcgError):
        B.Batch([S.laplacian_2d(8), S.laplacian_3d(4)])


# ------------------------------------------------------------------ Jacobi and mixed precision

def diag_of(P):
    c = S.to_csr(P) if P.layout != S.CSR32 else P
    rows = np.repeat(np.arange(c.n), np.diff(c.row_ptr))
    d = np.zeros(c.n)
    np.add.at(d, rows[c.col == rows], c.val[c.col == rows])
    return d


def test_batch_jacobi_first_iterations_vs_oracle(B):
    probs, bs = var2d_batch(k=6, seed=3)
    with B.Batch(probs, flags=B.PCG_JACOBI) as bt:
        xs, it, st, tr = bt.solve(bs, [1.0] * len(probs), tol=0.0, maxit=15)
    for P, b, x, i in zip(probs, bs, xs, it):
        o = oracle.pcg_sh(P, b, sigma=1.0, maxit=15, minv=1.0 / diag_of(P), log_every=0)
        assert i == o.iters
        assert np.linalg.norm(x - o.x) <= 1e-9 * np.linalg.norm(o.x)


def test_batch_jacobi_matches_single_solver(B):
    probs, bs = var2d_batch(k=8, seed=5)
    with B.Batch(probs, flags=B.PCG_JACOBI) as bt:
        xs, it, st, tr = bt.solve(bs, [1.0] * len(probs), tol=1e-9, maxit=5000)
    for P, b, x, i, code in zip(probs, bs, xs, it, st):
        with B.Solver(P, flags=B.PCG_JACOBI) as one:
            r = one.solve(b, method="spcg", sigma=1.0, tol=1e-9, maxit=5000)
        assert code == B.PCG_OK and r.status == B.PCG_OK
        assert abs(int(i) - r.iters) <= 0.02 * r.iters + 2
        assert np.linalg.norm(b - oracle.apply(P, x)) <= 3e-9 * np.linalg.norm(b)


MIXED_CASES = [
    ("var2d_jacobi", lambda: var2d_batch(k=10, seed=7), True, 1.0),
    ("lapl3d_identity", lambda: ([S.laplacian_3d(n, n + 3, n - 2) for n in (6, 11, 17, 24)],
                                 [S.normal(40 + i, n * (n + 3) * (n - 2)) for i, n in enumerate((6, 11, 17, 24))]),
     False, 6.0),
    ("csr_jacobi", lambda: ([S.random_sdd_csr(n, seed=n) for n in (500, 2003, 7001)],
                            [S.normal(50 + i, n) for i, n in enumerate((500, 2003, 7001))]), True, 1.0),
]


@pytest.mark.parametrize("name,maker,jac,sigma", MIXED_CASES, ids=[c[0] for c in MIXED_CASES])
def test_batch_mixed_reaches_tolerance(B, name, maker, jac, sigma):
    """Mixed precision with restarts in the batched launch: every system reaches 1e-8 in the
    binary64 true residual, recomputed here by the oracle's operator."""
    probs, bs = maker()
    with B.Batch(probs, flags=B.PCG_JACOBI if jac else 0, precision=B.PCG_MIXED_IR) as bt:
        xs, it, st, tr = bt.solve(bs, [sigma] * len(probs), tol=1e-8, maxit=20000)
    assert np.all(st == B.PCG_OK), st
    for P, b, x, t in zip(probs, bs, xs, tr):
        tt = np.linalg.norm(b - oracle.apply(P, x)) / np.linalg.norm(b)
        assert tt <= 1e-8 and abs(t - tt) <= 1e-6 * tt + 1e-16


def test_batch_mixed_matches_single_mixed(B):
    """The batch's mixed-precision solves (inner tolerance eta = 2^-14 by default) take the
    iterations of the single-system solver run with the same eta."""
    from paper_1706_05988_gb300 import pcg as C
    probs, bs = var2d_batch(k=5, seed=9)
    with B.Batch(probs, flags=B.PCG_JACOBI, precision=B.PCG_MIXED_IR) as bt:
        xs, it, st, tr = bt.solve(bs, [1.0] * len(probs), tol=1e-9, maxit=20000)
    for P, b, x, i, code in zip(probs, bs, xs, it, st):
        with B.Solver(P, flags=B.PCG_JACOBI) as one:
            assert C.pcg_set_param(one.ctx, C.PCG_PARAM_MIXED_ETA, 2.0 ** -14) == B.PCG_OK
            r = one.solve(b, method="spcg", sigma=1.0, tol=1e-9, maxit=20000, precision=B.PCG_MIXED_IR)
        assert code == B.PCG_OK and r.status == B.PCG_OK
        assert abs(int(i) - r.iters) <= 0.05 * r.iters + 10, (int(i), r.iters)
        assert np.linalg.norm(x - r.x) <= 1e-5 * np.linalg.norm(r.x)


def test_batch_jacobi_rejects_zero_diagonal(B):
    from paper_1706_05988_gb300 import pcg as C
    P = S.Problem(layout=S.CSR32, nx=0, ny=0, nz=0, row_ptr=np.array([0, 1, 2], dtype=np.int32),
                  col=np.array([1, 0], dtype=np.int32), val=np.array([1.0, 1.0]), n_csr=2)
    with pytest.raises(C.PcgError):
        B.Batch([P], flags=B.PCG_JACOBI)
    with B.Batch([S.laplacian_2d(8)]) as bt:
        assert bt.set_precision(7) == B.PCG_EINVAL
        assert bt.set_param(C.PCG_PARAM_MIXED_ETA, 2.0) == B.PCG_EINVAL
        assert bt.set_param(C.PCG_PARAM_MAX_RESTARTS, 3) == B.PCG_OK


def test_batch_size_classes_after_autotune(B):
    """Systems in all three size classes (n from 400 to 90,000) run concurrently, each class with
    the cluster size the autotuner picked for it; every result matches the single-system solver.
    Cluster sizes and kernel variants set per class by hand give new graphs whose results
    also converge, bit-identical between the two variants."""
    sides = [20, 33, 47, 64, 90, 120, 181, 256, 300]
    probs = [S.laplacian_2d(L, L + 3) for L in sides]
    bs = [S.normal(300 + i, P.n) for i, P in enumerate(probs)]
    sig = [4.0] * len(probs)
    with B.Batch(probs) as bt:
        c, ms = bt.autotune(bs, sig, probe_iters=30)
        assert c in (1, 2, 4, 8, 16) and np.isfinite(ms).any()
        nsys, csz, occ = bt.classes()
        assert nsys.tolist() == [4, 3, 2]                # n < 8192, < 65536, larger
        assert all(int(k) in (1, 2, 4, 8, 16) for k in csz)
        assert all(int(k) in (2, 4) for k in occ)       # the autotuner's kernel variant per class
        xs, it, st, tr = bt.solve(bs, sig, tol=1e-9, maxit=20000)
        xs2, it2, _, _ = bt.solve(bs, sig, tol=1e-9, maxit=20000)      # the graph replayed
        assert bt.set_class_cluster(3, 2) == B.PCG_EINVAL
        assert bt.set_class_cluster(0, 3) == B.PCG_EINVAL
        assert bt.set_class_occupancy(0, 3) == B.PCG_EINVAL
        assert bt.set_class_occupancy(3, 2) == B.PCG_EINVAL
        for k, cs in enumerate((1, 4, 16)):
            assert bt.set_class_cluster(k, cs) == B.PCG_OK
        assert bt.classes()[1].tolist() == [1, 4, 16]
        runs = []
        for occ in ((2, 4, 2), (4, 2, 4)):               # both kernel variants in every class
            for k, o in enumerate(occ):
                assert bt.set_class_occupancy(k, o) == B.PCG_OK
            assert bt.classes()[2].tolist() == list(occ)
            runs.append(bt.solve(bs, sig, tol=1e-9, maxit=20000))      # a new graph each
    for xs3, it3, st3, _ in runs:
        assert np.all(st3 == B.PCG_OK)
        for P, b, x in zip(probs, bs, xs3):
            assert np.linalg.norm(b - oracle.apply(P, x)) <= 3e-9 * np.linalg.norm(b)
    # the variant changes registers, not arithmetic: the same iterates
    assert np.array_equal(runs[0][1], runs[1][1])
    for x0, x1 in zip(runs[0][0], runs[1][0]):
        assert np.array_equal(x0, x1)
    assert np.all(st == B.PCG_OK)
    for P, b, x, x2, i, i2 in zip(probs, bs, xs, xs2, it, it2):
        assert i == i2 and np.array_equal(x, x2)
        with B.Solver(P) as one:
            r = one.solve(b, method="spcg", sigma=4.0, tol=1e-9, maxit=20000)
        assert abs(int(i) - r.iters) <= 0.02 * r.iters + 2
        assert np.linalg.norm(b - oracle.apply(P, x)) <= 3e-9 * np.linalg.norm(b)


def test_batch_mixed_wide_sweeps(B):
    """Row lengths that are multiples of 4 and of 2 (the binary32 sweeps then take four or two
    unknowns per thread) and odd ones in one mixed-precision batch, M = I and Jacobi."""
    dims = [(64, 40), (66, 31), (45, 45), (128, 17), (30, 30)]
    probs = [S.varcoef_2d(a, b, seed=60 + i) for i, (a, b) in enumerate(dims)]
    bs = [S.normal(400 + i, P.n) for i, P in enumerate(probs)]
    for jac in (False, True):
        sig = [1.0] * len(probs) if jac else [0.5 * float(np.median(P.diag)) for P in probs]
        with B.Batch(probs, flags=B.PCG_JACOBI if jac else 0, precision=B.PCG_MIXED_IR) as bt:
            xs, it, st, tr = bt.solve(bs, sig, tol=1e-8, maxit=50000)
        for P, b, x, code in zip(probs, bs, xs, st):
            assert code == B.PCG_OK
            assert np.linalg.norm(b - oracle.apply(P, x)) <= 1e-8 * np.linalg.norm(b)


FAMILIES = {
    "lapl2d": lambda: [S.laplacian_2d(40, 30), S.laplacian_2d(64, 20), S.laplacian_2d(17, 33)],
    "var2d": lambda: [S.varcoef_2d(a, b, lo_exp=-1.0, hi_exp=1.0, seed=81 + i)
                      for i, (a, b) in enumerate(((40, 30), (64, 20), (17, 33)))],
    "lapl3d": lambda: [S.laplacian_3d(12), S.laplacian_3d(16), S.laplacian_3d(9)],
    "var3d": lambda: [S.varcoef_3d(n, block=4, lo_exp=-1.0, hi_exp=1.0, seed=84 + n) for n in (12, 16)],
    "csr": lambda: [S.random_sdd_csr(n, seed=n) for n in (700, 1500)],
}


@pytest.mark.parametrize("family", list(FAMILIES))
def test_register_variants_agree(B, family):
    """Every operator family and every form (binary64 or mixed, M = I or Jacobi) through the
    batch kernel compiled for 2 and for 4 resident blocks per SM: bit-identical iterates,
    each near its tolerance against the oracle's operator (coefficient contrast 10^[-1, 1],
    at which the binary32 sweeps without Jacobi still converge)."""
    from paper_1706_05988_gb300 import pcg as C
    probs = FAMILIES[family]()
    bs = [S.normal(500 + i, P.n) for i, P in enumerate(probs)]
    for jac in (False, True):
        for prec in (C.PCG_FP64, C.PCG_MIXED_IR):
            sig = [1.0] * len(probs) if jac else [shift(P) for P in probs]
            runs = []
            with B.Batch(probs, flags=B.PCG_JACOBI if jac else 0, precision=prec) as bt:
                for occ in (2, 4):
                    for k in range(3):
                        assert bt.set_class_occupancy(k, occ) == B.PCG_OK
                    runs.append(bt.solve(bs, sig, tol=1e-8, maxit=20000))
            (x2, i2, s2, _), (x4, i4, s4, _) = runs
            assert np.all(s2 == B.PCG_OK) and np.array_equal(s2, s4), (jac, prec, s2, s4)
            assert np.array_equal(i2, i4), (jac, prec)
            for P, b, a, c in zip(probs, bs, x2, x4):
                assert np.array_equal(a, c)
                assert np.linalg.norm(b - oracle.apply(P, a)) <= 3e-8 * np.linalg.norm(b)

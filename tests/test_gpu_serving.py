"""Continuous-batching server (pcg_server_create / pcg_submit / pcg_poll), GB300 only.

A request's result is the same bit for bit whether it runs alone or among other
requests (each request is solved by one cluster with a fixed reduction order), every
result reaches its tolerance by the oracle's true residual, requests wait for arena
memory and still complete, and an idle server restarts its kernel for new work."""
import threading
import time

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


def random_sdd(n, seed):
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    deg = rng.integers(3, 13, size=n)
    rows = np.repeat(np.arange(n), deg)
    cols = rng.integers(0, n, size=rows.size)
    keep = rows != cols
    U = sp.coo_matrix((-rng.random(keep.sum()), (rows[keep], cols[keep])), shape=(n, n)).tocsr()
    A = (U + U.T).tocsr()
    A.sum_duplicates()
    d = np.asarray(np.abs(A).sum(axis=1)).ravel() * 1.01 + 1e-3
    A = (A + sp.diags(d)).tocsr()
    A.sort_indices()
    return S.Problem(S.CSR32, row_ptr=A.indptr.astype(np.int32), col=A.indices.astype(np.int32),
                     val=A.data.astype(np.float64), n_csr=n)


def request_mix():
    probs = [S.laplacian_2d(40, 33), S.laplacian_3d(18, 15, 12), S.varcoef_2d(30, 30, seed=4),
             random_sdd(3000, 1), S.laplacian_2d(7, 5), S.varcoef_3d(16, block=4, lo_exp=-1.0, hi_exp=1.0, seed=2), random_sdd(500, 2),
             S.laplacian_3d(25)]
    bs = [S.normal(50 + i, P.n) for i, P in enumerate(probs)]
    return probs, bs


def wait(srv, t, timeout=60.0):
    t0 = time.time()
    while True:
        r = srv.poll(t)
        if r is not None:
            return r
        assert time.time() - t0 < timeout, "request did not finish"
        time.sleep(0.0005)


def test_same_result_alone_and_in_the_mix(B):
    probs, bs = request_mix()
    alone = []
    for P, b in zip(probs, bs):
        with B.Server(256 << 20, 4) as srv:
            alone.append(wait(srv, srv.submit(P, b, tol=1e-10)))
    with B.Server(256 << 20, 16) as srv:
        tickets = [srv.submit(P, b, tol=1e-10) for P, b in zip(probs, bs)]
        mixed = [wait(srv, t) for t in reversed(tickets)][::-1]
    for P, b, a, m in zip(probs, bs, alone, mixed):
        assert a[0] == m[0] and a[2] == m[2] and np.array_equal(a[1], m[1])
        assert m[0] == B.PCG_OK
        tr = np.linalg.norm(b - oracle.apply(P, m[1])) / np.linalg.norm(b)
        assert tr <= 2e-10 and abs(tr - m[3]) <= 1e-6 * tr + 1e-16


def test_matches_single_system_solver(B):
    P = S.varcoef_2d(45, 31, seed=9)
    b = S.normal(9, P.n)
    sigma = float(np.mean(P.diag))
    with B.Server(64 << 20, 2) as srv:
        st, x, it, tr = wait(srv, srv.submit(P, b, tol=1e-9, sigma=sigma))
    with B.Solver(P) as one:
        r = one.solve(b, method="spcg", sigma=sigma, tol=1e-9, maxit=100000)
    assert st == r.status == B.PCG_OK and abs(it - r.iters) <= 0.02 * r.iters + 2
    assert np.linalg.norm(x - r.x) <= 1e-4 * np.linalg.norm(r.x)


def test_admission_waits_for_memory(B):
    probs = [S.laplacian_3d(40) for _ in range(6)]          # ~4.1 MB of vectors each
    bs = [S.normal(i, P.n) for i, P in enumerate(probs)]
    with B.Server(10 << 20, 8) as srv:                        # room for two at a time
        tickets = [srv.submit(P, b, tol=1e-8) for P, b in zip(probs, bs)]
        waiting, inflight, free = srv.stats()
        assert waiting >= 3 and inflight <= 2
        res = [wait(srv, t) for t in tickets]
        assert srv.stats()[:2] == (0, 0)
    for P, b, r in zip(probs, bs, res):
        assert r[0] == B.PCG_OK
        assert np.linalg.norm(b - oracle.apply(P, r[1])) <= 2e-8 * np.linalg.norm(b)


def test_idle_kernel_restarts(B):
    P, b, _ = S.poisson2d_manufactured(50)
    with B.Server(32 << 20, 2) as srv:
        first = wait(srv, srv.submit(P, b, tol=1e-10))
        time.sleep(0.2)                                       # the kernel exits after 20 ms idle
        second = wait(srv, srv.submit(P, b, tol=1e-10))
    assert first[0] == second[0] == B.PCG_OK and np.array_equal(first[1], second[1])


def test_submissions_from_two_threads(B):
    probs, bs = request_mix()
    out = {}
    with B.Server(256 << 20, 8) as srv:
        def worker(idx):
            for i in idx:
                out[i] = wait(srv, srv.submit(probs[i], bs[i], tol=1e-9))
        th = [threading.Thread(target=worker, args=(list(range(k, len(probs), 2)),)) for k in (0, 1)]
        for t in th:
            t.start()
        for t in th:
            t.join()
    assert sorted(out) == list(range(len(probs))) and all(v[0] == B.PCG_OK for v in out.values())


def test_server_rejects_bad_requests(B):
    from paper_1706_05988_gb300 import pcg as C
    with B.Server(1 << 20, 1) as srv:
        with pytest.raises(C.PcgError):
            srv.submit(S.laplacian_3d(64), np.ones(64 ** 3))     # can never fit in 1 MiB
        with pytest.raises(C.PcgError):
            srv.submit(S.laplacian_2d(8), np.ones(64), method=C.PCG_CG)
    with pytest.raises(C.PcgError):
        B.Server(100, 1)


# ------------------------------------------------------------------ mixed precision and Jacobi

MODES = [(0, 0), ("jac", 0), (0, "mixed"), ("jac", "mixed")]


def _mode(B, jac, prec):
    return (B.PCG_JACOBI if jac else 0), (B.PCG_MIXED_IR if prec else B.PCG_FP64)


def test_mixed_jacobi_alone_and_in_the_mix(B):
    """Requests of all four kinds (binary64 / mixed, M = I / Jacobi) in one stream: each result
    is bit-identical to the same request served alone and reaches its tolerance."""
    probs, bs = request_mix()
    kinds = [MODES[i % 4] for i in range(len(probs))]
    alone = []
    for P, b, (jac, prec) in zip(probs, bs, kinds):
        fl, pr = _mode(B, jac, prec)
        with B.Server(256 << 20, 4) as srv:
            alone.append(wait(srv, srv.submit(P, b, tol=1e-9, flags=fl, precision=pr)))
    with B.Server(256 << 20, 16) as srv:
        tickets = []
        for P, b, (jac, prec) in zip(probs, bs, kinds):
            fl, pr = _mode(B, jac, prec)
            tickets.append(srv.submit(P, b, tol=1e-9, flags=fl, precision=pr))
        mixed = [wait(srv, t) for t in tickets]
    for P, b, a, m in zip(probs, bs, alone, mixed):
        assert a[0] == m[0] and a[2] == m[2] and np.array_equal(a[1], m[1])
        assert m[0] == B.PCG_OK
        tr = np.linalg.norm(b - oracle.apply(P, m[1])) / np.linalg.norm(b)
        assert tr <= 2e-9 and abs(tr - m[3]) <= 1e-6 * tr + 1e-16


def test_served_modes_match_batch(B):
    """A served request and the same system in a batch run the same per-cluster solver (an odd
    row length: the batched mixed sweep then also takes one unknown per thread)."""
    P = S.varcoef_2d(45, 38, seed=11)
    b = S.normal(12, P.n)
    for jac, prec in MODES:
        fl, pr = _mode(B, jac, prec)
        with B.Server(64 << 20, 2) as srv:
            st, x, it, tr = wait(srv, srv.submit(P, b, tol=1e-9, sigma=1.0 if jac else 2.0, flags=fl, precision=pr))
        with B.Batch([P], flags=fl, precision=pr) as bt:
            assert bt.set_cluster(2) == B.PCG_OK
            xs, its, sts, trs = bt.solve([b], [1.0 if jac else 2.0], tol=1e-9, maxit=100000)
        assert st == sts[0] == B.PCG_OK and it == its[0] and np.array_equal(x, xs[0]), (jac, prec)


def test_submit_ex_rejects_bad_modes(B):
    from paper_1706_05988_gb300 import pcg as C
    with B.Server(16 << 20, 2) as srv:
        with pytest.raises(C.PcgError):
            srv.submit(S.laplacian_2d(8), np.ones(64), flags=0x4000)
        with pytest.raises(C.PcgError):
            srv.submit(S.laplacian_2d(8), np.ones(64), precision=9)


def dense_rows_sdd(n, per_row, seed):
    """SDD CSR with many entries per row (a request whose staging is large)."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(n), per_row)
    cols = rng.integers(0, n, size=rows.size)
    keep = rows != cols
    U = sp.coo_matrix((-rng.random(keep.sum()), (rows[keep], cols[keep])), shape=(n, n)).tocsr()
    A = (U + U.T).tocsr()
    A.sum_duplicates()
    d = np.asarray(np.abs(A).sum(axis=1)).ravel() * 1.01 + 1e-3
    A = (A + sp.diags(d)).tocsr()
    A.sort_indices()
    return S.Problem(S.CSR32, row_ptr=A.indptr.astype(np.int32), col=A.indices.astype(np.int32),
                     val=A.data.astype(np.float64), n_csr=n)


def test_waiting_request_keeps_its_own_copy(B):
    """A request that has to wait for memory copies its arrays at submission: the caller may
    overwrite them at once.  A request whose host data is too large for the staging ring takes
    the direct path.  Both results solve the systems as submitted."""
    import copy
    first = S.laplacian_2d(400, 400)                   # 10.3 MB of arena, staged
    big = dense_rows_sdd(10000, 60, 5)                 # 14.4 MB of arena, 13.9 MB of host data > 12 MB ring
    b1, b2 = S.normal(90, first.n), S.normal(91, big.n)
    orig = [(first, b1.copy()), (copy.deepcopy(big), b2.copy())]
    with B.Server(24 << 20, 4) as srv:
        t1 = srv.submit(first, b1, tol=1e-10)
        t2 = srv.submit(big, b2, tol=1e-10)            # waits: both do not fit in 24 MB
        b1[:] = 7.0                                    # the caller reuses its buffers
        b2[:] = -3.0
        big.val[:] = 1.0
        r1 = wait(srv, t1)
        r2 = wait(srv, t2)
    for (P, b), r in zip(orig, (r1, r2)):
        assert r[0] == B.PCG_OK
        assert np.linalg.norm(b - oracle.apply(P, r[1])) <= 2e-10 * np.linalg.norm(b)


def test_device_lane_requests(B):
    """Requests of n >= 2^19 run on the whole GPU through the single-system solver while the
    cluster lanes pause; small requests submitted around them still complete, and every
    result solves its system."""
    big3d = S.laplacian_3d(81)                                   # n = 531,441
    big2d = S.varcoef_2d(800, 700, lo_exp=-1.0, hi_exp=1.0, seed=3)   # n = 560,000
    small = [S.laplacian_2d(40, 30), random_sdd(2000, 7), S.laplacian_3d(15)]
    reqs = [(big3d, S.normal(70, big3d.n), 0, B.PCG_FP64), (small[0], S.normal(71, small[0].n), 0, B.PCG_FP64),
            (big2d, S.normal(72, big2d.n), B.PCG_JACOBI, B.PCG_MIXED_IR),
            (small[1], S.normal(73, small[1].n), B.PCG_JACOBI, B.PCG_MIXED_IR),
            (small[2], S.normal(74, small[2].n), 0, B.PCG_FP64)]
    with B.Server(256 << 20, 8) as srv:
        tickets = [srv.submit(P, b, tol=1e-8, flags=fl, precision=pr) for P, b, fl, pr in reqs]
        out = [wait(srv, t, timeout=120.0) for t in tickets]
    for (P, b, fl, pr), r in zip(reqs, out):
        assert r[0] == B.PCG_OK, r[0]
        tr = np.linalg.norm(b - oracle.apply(P, r[1])) / np.linalg.norm(b)
        assert tr <= (1e-8 if pr == B.PCG_MIXED_IR else 3e-8) and abs(tr - r[3]) <= 1e-3 * tr + 1e-15, (tr, r[3])


def test_smaller_requests_go_first(B):
    """Small requests that arrive while a whole-GPU request runs are taken by the cluster
    lanes before the next whole-GPU request starts: they finish before it."""
    d1 = S.laplacian_2d(1448)                                    # n = 2,096,704: runs long enough
    d2 = S.laplacian_3d(81)                                      # to hold the small submissions
    small = [S.laplacian_2d(30, 20), random_sdd(1500, 11), S.laplacian_3d(12), S.laplacian_2d(64),
             random_sdd(800, 12), S.laplacian_3d(20, 18, 9)]
    reqs = [(d1, S.normal(80, d1.n), 1e-10)]
    reqs += [(P, S.normal(82 + i, P.n), 1e-8) for i, P in enumerate(small)]
    reqs += [(d2, S.normal(81, d2.n), 1e-8)]
    with B.Server(256 << 20, 16) as srv:
        t0 = time.time()
        pending, fin, res = {}, {}, {}

        def poll_all():
            for t in list(pending):
                r = srv.poll(t)
                if r is not None:
                    k = pending.pop(t)
                    fin[k], res[k] = time.time(), r

        for k, (P, b, tol) in enumerate(reqs):
            if k == 1:                                           # d1 taken by a solving thread
                while srv.stats()[0] > 0:
                    assert time.time() - t0 < 60.0
                    time.sleep(0.001)
                time.sleep(0.01)
            if k == len(reqs) - 1:
                time.sleep(0.05)                                 # the small requests' copies land
                poll_all()
            pending[srv.submit(P, b, tol=tol)] = k
        while pending:
            assert time.time() - t0 < 120.0, "requests did not finish"
            poll_all()
            time.sleep(0.0005)
    for k, (P, b, tol) in enumerate(reqs):
        assert res[k][0] == B.PCG_OK, (k, res[k][0])
        tr = np.linalg.norm(b - oracle.apply(P, res[k][1])) / np.linalg.norm(b)
        assert tr <= 3 * tol, (k, tr)
    last = len(reqs) - 1
    assert fin[0] < fin[last]                                     # the second whole-GPU request waits
    assert max(fin[k] for k in range(1, last)) < fin[last]        # the small ones before it


def test_two_whole_gpu_requests_at_once(B):
    """Two whole-GPU requests submitted together are solved side by side; both results
    solve their systems."""
    reqs = [(S.laplacian_2d(1100), S.normal(90, 1100 * 1100), 1e-9, B.PCG_FP64),
            (S.laplacian_3d(84), S.normal(91, 84 ** 3), 1e-9, B.PCG_MIXED_IR),
            (S.varcoef_2d(760, 700, lo_exp=-1.0, hi_exp=1.0, seed=5), S.normal(92, 760 * 700), 1e-8, B.PCG_FP64)]
    with B.Server(256 << 20, 8) as srv:
        tickets = [srv.submit(P, b, tol=tol, precision=pr) for P, b, tol, pr in reqs]
        out = [wait(srv, t, timeout=120.0) for t in tickets]
    for (P, b, tol, pr), r in zip(reqs, out):
        assert r[0] == B.PCG_OK, r[0]
        tr = np.linalg.norm(b - oracle.apply(P, r[1])) / np.linalg.norm(b)
        assert tr <= 3 * tol and abs(tr - r[3]) <= 1e-3 * tr + 1e-15, (tr, r[3])


def test_destroy_with_whole_gpu_requests_in_flight(B):
    """Destroying a server while whole-GPU requests are being prepared, solved or wait,
    and small ones are queued, returns (their contexts are freed) and leaves the GPU
    usable: a new server then solves a request."""
    big = [S.laplacian_2d(1200), S.laplacian_3d(90), S.laplacian_2d(800, 700), random_sdd(600_000, 13)]
    small = [S.laplacian_2d(40, 30), random_sdd(2000, 14)]
    t0 = time.time()
    with B.Server(256 << 20, 8) as srv:
        for i, P in enumerate(big + small):
            srv.submit(P, S.normal(100 + i, P.n), tol=1e-10)
        time.sleep(0.05)                                  # some are running, some prepared or queued
    assert time.time() - t0 < 60.0
    P = S.laplacian_3d(20)
    b = S.normal(110, P.n)
    with B.Server(64 << 20, 2) as srv:
        st, x, it, tr = wait(srv, srv.submit(P, b, tol=1e-9))
    assert st == B.PCG_OK and np.linalg.norm(b - oracle.apply(P, x)) <= 2e-9 * np.linalg.norm(b)

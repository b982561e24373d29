"""Host-side pieces of bench.py that need no GPU: the serving trace and the oracle's timed
samples beside the side measurements."""
import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
import synthetic as S  # noqa: E402


def test_serving_trace_prefix_is_the_same_stream():
    full = bench.serving_trace(40, 2000.0, n_max_exp=3.5)
    head = bench.serving_trace(40, 2000.0, n_max_exp=3.5, first=6)
    assert len(head) == 6
    for (a0, P0, b0, t0), (a1, P1, b1, t1) in zip(full, head):
        assert a0 == a1 and t0 == t1 and P0.n == P1.n and np.array_equal(b0, b1)
    arr = np.array([r[0] for r in full])
    assert np.all(np.diff(arr) > 0)
    tols = np.array([r[3] for r in full])
    assert np.all((tols >= 1e-10) & (tols <= 1e-6))


def test_request_sigma():
    assert bench.request_sigma(S.laplacian_2d(8)) == 4.0
    assert bench.request_sigma(S.laplacian_3d(5)) == 6.0
    P = S.random_sdd_csr(300, seed=1)
    d = np.array([P.val[P.row_ptr[i]:P.row_ptr[i + 1]][P.col[P.row_ptr[i]:P.row_ptr[i + 1]] == i].sum()
                  for i in range(P.n)])
    assert abs(bench.request_sigma(P) - d.mean()) <= 1e-12 * d.mean()


def test_cpu_side_baselines_small():
    a = argparse.Namespace(batch_systems=8, batch_side_max=40, no_serving=False, serving_requests=30,
                           serving_small_requests=30, serving_rate=2000.0, serving_n_max_exp=3.3)
    work = 8 * 1000 * 100.0
    out = bench.cpu_side_baselines(S, a, {"fp64_jacobi": {"unknown_iterations": work}}, None)
    bt = out["batch_fp64_jacobi"]
    assert bt["solves_per_s"] > 0 and bt["est_batch_s"] > 0
    assert abs(bt["solves_per_s"] * bt["est_batch_s"] - 8) < 1e-9
    sv = out["serving_n_le_1e5_fp64"]
    assert sv["solves_per_s"] > 0 and "requests back to back" in sv["sample"]
    assert "varcoef_128_fp64_jacobi" not in out


def test_request_policy():
    """served_mixed: mixed precision everywhere, Jacobi only on CSR; fp64: binary64, M = I."""
    from paper_1706_05988_gb300 import pcg as C
    lap, csr = S.laplacian_2d(10), S.random_sdd_csr(50, seed=2)
    assert bench.request_policy(lap, "fp64") == (0, C.PCG_FP64)
    assert bench.request_policy(lap, "mixed") == (0, C.PCG_MIXED_IR)
    assert bench.request_policy(csr, "mixed") == (C.PCG_JACOBI, C.PCG_MIXED_IR)
    assert bench.request_policy(lap, "mixed_jacobi") == (C.PCG_JACOBI, C.PCG_MIXED_IR)

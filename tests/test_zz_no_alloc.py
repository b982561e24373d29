"""pcg_true_residual_noalloc, the allocation-free entry point (GB300 only).

It serves callers that must not allocate device memory (see include/pcg.h).
It is checked against the solver's own true residual (pcg_solve_device reports
||b - A x|| at exit) and against pcg_apply, on two calls in a row, since every
call reuses the same file-scope scratch.  This file is collected last, so a run
that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

TOL = 1e-10          # relative tolerance of the FP64 GPU comparisons in these tests


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1706_05988_gb300 import build
    build.build()
    import paper_1706_05988_gb300 as pkg
    return pkg


def device_matrix(P):
    """pcg_matrix with device arrays (what the entry point requires) and the tensors behind it."""
    import torch
    from paper_1706_05988_gb300 import pcg as C
    keep = {}
    if P.layout == S.CSR32:
        keep = {"row_ptr": torch.from_numpy(P.row_ptr).cuda(), "col": torch.from_numpy(P.col).cuda(),
                "val": torch.from_numpy(P.val).cuda()}
    elif not P.constant:
        keep = {k: torch.from_numpy(getattr(P, k)).cuda() for k in ("diag", "ax", "ay", "az")}
    return C.Matrix(P, device_arrays=keep if keep else {}), keep


PROBLEMS = [("lapl3d_48", lambda: S.laplacian_3d(48)),
            ("varcoef3d_24", lambda: S.varcoef_3d(24, block=8, seed=1)),
            ("lapl2d_odd", lambda: S.laplacian_2d(63, 41)),
            ("csr_lapl3d", lambda: S.to_csr(S.laplacian_3d(20, 18, 16)))]


@pytest.mark.parametrize("name,maker", PROBLEMS, ids=[p[0] for p in PROBLEMS])
def test_noalloc_matches_solver_twice(B, name, maker):
    import torch
    from paper_1706_05988_gb300 import pcg as C
    P = maker()
    b = torch.from_numpy(S.normal(3, P.n)).cuda()
    bn = float(torch.linalg.vector_norm(b))
    with B.Solver(P) as s:
        x = torch.empty_like(b)
        res = C.pcg_result()
        st = C.pcg_solve_device(s.ctx, b, None, C.PCG_SPCG, 1.0, 0.0, 30, C.PCG_FP64, x, res)
        assert st == C.PCG_ENOTCONV
        ref_true = res.final_true_relres * bn          # ||b - A x|| from the solver's exit check
        ax = torch.empty_like(b)
        assert C.pcg_apply(s.ctx, x, ax) == C.PCG_OK
    r = torch.from_numpy(S.normal(5, P.n)).cuda()
    ref_gap = float(torch.linalg.vector_norm((b - ax) - r))
    M, keep = device_matrix(P)
    outs = []
    for _ in range(2):
        norms = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        assert C.pcg_true_residual_noalloc(M.m, b, x, r, norms) == C.PCG_OK
        torch.cuda.synchronize()
        outs.append(norms.cpu().numpy())
    for o in outs:
        assert abs(o[0] - ref_true) <= TOL * ref_true, (o[0], ref_true)
        assert abs(o[1] - ref_gap) <= TOL * ref_gap, (o[1], ref_gap)
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_without_r_and_limits(B):
    import torch
    from paper_1706_05988_gb300 import pcg as C
    P = S.laplacian_3d(16)
    b = torch.from_numpy(S.normal(1, P.n)).cuda()
    x = torch.zeros_like(b)
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    M, _ = device_matrix(P)
    assert C.pcg_true_residual_noalloc(M.m, b, x, None, norms) == C.PCG_OK
    torch.cuda.synchronize()
    o = norms.cpu().numpy()
    assert abs(o[0] - float(torch.linalg.vector_norm(b))) <= TOL * o[0] and np.isnan(o[1])
    # beyond the stated maximum: rejected before any work is queued
    big = S.laplacian_3d(257, 256, 256)
    assert big.n > 16777216
    Mb, _ = device_matrix(big)
    assert C.pcg_true_residual_noalloc(Mb.m, b, x, None, norms) == C.PCG_EINVAL
    # misaligned vectors are rejected (128-bit loads)
    assert C.pcg_true_residual_noalloc(M.m, b[1:], x[1:], None, norms) == C.PCG_EINVAL


def test_noalloc_misaligned_pointers_rejected(B):
    """8-byte misaligned vectors or norms are rejected with PCG_EINVAL before any CUDA call,
    on both the two-unknowns-per-thread path (even row length) and the one-unknown path."""
    import torch
    from paper_1706_05988_gb300 import pcg as C
    for P in (S.laplacian_3d(16), S.laplacian_2d(63, 41)):
        b = torch.from_numpy(S.normal(1, P.n + 1)).cuda()
        x = torch.zeros_like(b)
        norms = torch.zeros(3, dtype=torch.float64, device="cuda")
        M, _ = device_matrix(P)
        assert C.pcg_true_residual_noalloc(M.m, b, x, None, norms) == C.PCG_OK
        assert C.pcg_true_residual_noalloc(M.m, b, x, None, norms.data_ptr() + 4) == C.PCG_EINVAL
        assert C.pcg_true_residual_noalloc(M.m, b.data_ptr() + 4, x, None, norms) == C.PCG_EINVAL
        assert C.pcg_true_residual_noalloc(M.m, b, x, x.data_ptr() + 4, norms) == C.PCG_EINVAL
        torch.cuda.synchronize()


def test_noalloc_at_the_limit_on_a_side_stream(B):
    """n = PCG_NOALLOC_MAX_N (the 256^3 Laplacian): every partial slot is used and the last
    block sums all 4,096 of them.  Two calls on a non-default stream against the solver's
    exit true residual and a residual formed from pcg_apply."""
    import torch
    from paper_1706_05988_gb300 import pcg as C
    P = S.laplacian_3d(256)
    assert P.n == 16777216
    xs = torch.from_numpy(S.uniform_pm1(0, P.n)).cuda()
    with B.Solver(P) as s:
        ax = torch.empty_like(xs)
        assert C.pcg_apply(s.ctx, xs, ax) == C.PCG_OK
        b = ax.clone()
        bn = float(torch.linalg.vector_norm(b))
        x = torch.empty_like(b)
        res = C.pcg_result()
        st = C.pcg_solve_device(s.ctx, b, None, C.PCG_SPCG, 6.0, 0.0, 12, C.PCG_FP64, x, res)
        assert st == C.PCG_ENOTCONV
        ref_true = res.final_true_relres * bn
        assert C.pcg_apply(s.ctx, x, ax) == C.PCG_OK
    torch.cuda.synchronize()
    r = torch.from_numpy(S.normal(5, P.n)).cuda()
    ref_gap = float(torch.linalg.vector_norm((b - ax) - r))
    M, _ = device_matrix(P)
    side = torch.cuda.Stream()
    outs = []
    for _ in range(2):
        norms = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            assert C.pcg_true_residual_noalloc(M.m, b, x, r, norms, side.cuda_stream) == C.PCG_OK
        side.synchronize()
        outs.append(norms.cpu().numpy())
    for o in outs:
        assert abs(o[0] - ref_true) <= TOL * ref_true, (o[0], ref_true)
        assert abs(o[1] - ref_gap) <= TOL * ref_gap, (o[1], ref_gap)
    assert np.array_equal(outs[0], outs[1])

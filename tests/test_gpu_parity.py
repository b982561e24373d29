"""CUDA path vs the FP64 oracle, through the C ABI (GB300 only).

Tolerances (fixed by the method's target): alpha_i, beta_i within 1e-10
relative over the first 20 iterations; final true relative residual within a
factor 10 of the oracle's.  The two sides sum in different orders (the GPU
uses FMA and a two-level tree reduction), so nothing is compared bit for bit
except properties that are exact on the GPU side itself (determinism, the
sigma = 0 path, host vs device entry points).
"""
import numpy as np
import pytest

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu

TOL_SCALARS = 1e-10
N_SCALARS = 20


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1706_05988_gb300 import build
    build.build()
    import paper_1706_05988_gb300 as pkg
    return pkg


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def check_scalars(g, o, k=N_SCALARS, tol=TOL_SCALARS):
    k = min(k, len(o.alpha), len(g.alpha))
    assert k > 0
    assert rel(g.alpha[:k], o.alpha[:k]) <= tol, (g.alpha[:k], o.alpha[:k])
    assert rel(g.beta[1:k], o.beta[1:k]) <= tol
    assert g.beta[0] == 0.0


def check_final(g, o, bnorm):
    gt = g.final_true_relres
    ot = o.true[-1] / bnorm
    assert 0.1 * ot <= gt <= 10 * ot, (gt, ot)


def run_both(B, P, b, method, sigma, maxit, tol=0.0, x0=None, flags=0):
    with B.Solver(P, flags=flags) as s:
        g = s.solve(b, x0=x0, method=method, sigma=sigma, tol=tol, maxit=maxit, true_every=1)
    if method == "cg":
        o = oracle.cg(P, b, x0=x0, maxit=maxit, rtol=tol, log_every=1)
    else:
        o = oracle.pcg_sh(P, b, x0=x0, sigma=sigma if method == "spcg" else 0.0, maxit=maxit, rtol=tol, log_every=1)
    return g, o


# ---------------------------------------------------------------- 2D Poisson 100x100 (n = 10,000)

@pytest.mark.parametrize("method,sigma", [("cg", 0.0), ("pcg", 0.0), ("spcg", 4.0)])
def test_poisson2d_100(B, method, sigma):
    P, b, xs = S.poisson2d_manufactured(100)
    g, o = run_both(B, P, b, method, sigma, maxit=600)
    if method == "pcg":
        # unshifted p-CG loses its way after stagnating and stops on a non-positive 1/alpha; where exactly
        # depends on rounding (the oracle stops at 415), so compare the outcome, not the iteration count
        assert g.status == B.PCG_EBREAKDOWN and o.status == 2
        assert abs(g.iters - o.iters) <= 100
    else:
        assert g.iters == o.iters == 600
    check_scalars(g, o)
    check_final(g, o, np.linalg.norm(b))
    # recursive residual history follows the oracle's while far above rounding level
    k = min(len(g.rec), len(o.rec))
    m = o.rec[:k] > 1e-6 * o.rec[0]
    assert rel(g.rec[:k][m], o.rec[:k][m]) < 1e-4
    # true residual and gap histories are logged at every iteration
    assert np.all(np.isfinite(g.true)) and np.all(np.isfinite(g.gap))


def test_poisson2d_100_accuracy_ordering(B):
    """Attainable accuracy: CG and p-CG-sh reach ~1e-13 relative; the gap of p-CG-sh stays CG-like."""
    P, b, xs = S.poisson2d_manufactured(100)
    bn = np.linalg.norm(b)
    with B.Solver(P) as s:
        cg = s.solve(b, method="cg", maxit=2000, true_every=10)
        sh = s.solve(b, method="spcg", sigma=4.0, maxit=2000, true_every=10)
        pc = s.solve(b, method="pcg", maxit=2000, true_every=10)
    assert cg.final_true_relres < 1e-13
    assert sh.final_true_relres < 10 * cg.final_true_relres
    assert np.nanmax(sh.gap) / bn < 1e-12
    assert pc.final_true_relres > 3 * cg.final_true_relres   # p-CG loses accuracy (or breaks down)


# ---------------------------------------------------------------- lapl200 (Table 1)

def test_lapl200_table1(B):
    P, b = S.lapl200()
    with B.Solver(P) as s:
        cg = s.solve(b, method="cg", maxit=500)
        sh = s.solve(b, method="spcg", sigma=4.0, maxit=500)
    for r in (cg, sh):
        assert r.iters == 500
        assert 3e-12 <= r.final_true_relres <= 1.4e-11       # Table 1: 6.8e-12 (||b|| = 1)
    o = oracle.pcg_sh(P, b, sigma=4.0, maxit=500, log_every=0)
    check_scalars(sh, o)


# ---------------------------------------------------------------- operators and shapes

SHAPES = [
    ("2d_odd", lambda: S.laplacian_2d(37, 23)),
    ("2d_row", lambda: S.laplacian_2d(1, 9)),
    ("2d_col", lambda: S.laplacian_2d(64, 1)),
    ("3d_even", lambda: S.laplacian_3d(20, 18, 16)),
    ("3d_odd", lambda: S.laplacian_3d(15, 17, 9)),
    ("3d_flat", lambda: S.laplacian_3d(12, 10, 1)),
    ("var2d", lambda: S.varcoef_2d(48, 40, seed=1)),
    ("var2d_odd", lambda: S.varcoef_2d(33, 21, seed=2)),
    ("var3d", lambda: S.varcoef_3d(24, block=8, seed=3)),
    ("var3d_odd", lambda: S.varcoef_3d(17, block=4, seed=4)),
    ("csr_lapl3d", lambda: S.to_csr(S.laplacian_3d(18, 14, 10))),
    ("csr_var2d", lambda: S.to_csr(S.varcoef_2d(30, 26, seed=5))),
]


def shift_for(P):
    """A shift inside the spectrum: half the median diagonal entry."""
    c = S.to_csr(P)
    rows = np.repeat(np.arange(c.n), np.diff(c.row_ptr))
    return 0.5 * float(np.median(c.val[c.col == rows]))


@pytest.mark.parametrize("name,maker", SHAPES, ids=[s[0] for s in SHAPES])
@pytest.mark.parametrize("method", ["cg", "spcg"])
def test_shapes_vs_oracle(B, name, maker, method):
    """20 iterations: scalars and iterates.  High-contrast coefficients amplify rounding
    differences later on (the oracle against itself with b perturbed in the last bit moves
    x by ~1e-11 relative after 20 iterations but by up to 5e-3 after 60), so the iterate is
    compared at 20 iterations."""
    P = maker()
    b = S.normal(7, P.n)
    bn = np.linalg.norm(b)
    sigma = shift_for(P) if method == "spcg" else 0.0
    maxit = min(20, P.n)
    g, o = run_both(B, P, b, method, sigma, maxit)
    assert g.iters == o.iters
    live = int(np.sum(o.rec[:o.iters] > 1e-9 * o.rec[0]))
    if live > 0:
        check_scalars(g, o, k=live)
    if o.true[-1] > 1e-12 * bn:
        check_final(g, o, bn)
    else:
        assert g.final_true_relres < 1e-11
    assert np.linalg.norm(g.x - o.x) <= 1e-8 * np.linalg.norm(o.x)


@pytest.mark.parametrize("name,maker", [s for s in SHAPES if s[0] in ("2d_odd", "var2d_odd", "3d_odd", "csr_var2d")],
                         ids=["2d_odd", "var2d_odd", "3d_odd", "csr_var2d"])
def test_shapes_converged(B, name, maker):
    """Run to ||r|| <= 1e-10 ||b||: same stopping iteration (to a few percent) and true residual."""
    P = maker()
    b = S.normal(7, P.n)
    bn = np.linalg.norm(b)
    sigma = shift_for(P)
    g, o = run_both(B, P, b, "spcg", sigma, maxit=5000, tol=1e-10)
    assert g.status == B.PCG_OK and o.status == 1
    assert abs(g.iters - o.iters) <= 0.05 * o.iters + 2
    check_final(g, o, bn)


@pytest.mark.parametrize("maker", [lambda: S.laplacian_3d(20, 18, 16), lambda: S.laplacian_2d(37, 23)],
                         ids=["3d", "2d_odd"])
def test_fp64_sum_rows_vs_oracle(B, maker):
    """The FP64-addition stencil rows (PCG_STENCIL_FP64_SUM) against the oracle."""
    P = maker()
    b = S.normal(3, P.n)
    g, o = run_both(B, P, b, "spcg", shift_for(P), 20, flags=B.PCG_STENCIL_FP64_SUM)
    check_scalars(g, o)
    assert np.linalg.norm(g.x - o.x) <= 1e-8 * np.linalg.norm(o.x)


DOT_SHAPES = [s for s in SHAPES if s[0] in ("3d_even", "2d_odd", "var3d", "csr_var2d")]


@pytest.mark.parametrize("name,maker", DOT_SHAPES, ids=[s[0] for s in DOT_SHAPES])
def test_dot_forms_vs_oracle(B, name, maker):
    """The merged dots (r,r), (w,r) accumulated in binary64 (the default) and on the FP32 pipe
    (PCG_DOTS_SPLIT32: exact binary32 splits, TwoProd/TwoSum): both meet the parity bar against
    the oracle, and they agree with each other to 1e-12 over 20 iterations."""
    P = maker()
    b = S.normal(7, P.n)
    sigma = shift_for(P)
    g64, o = run_both(B, P, b, "spcg", sigma, 20)
    gff, _ = run_both(B, P, b, "spcg", sigma, 20, flags=B.PCG_DOTS_SPLIT32)
    check_scalars(g64, o)
    check_scalars(gff, o)
    assert rel(gff.alpha, g64.alpha) <= 1e-12 and rel(gff.beta[1:], g64.beta[1:]) <= 1e-12
    assert np.linalg.norm(gff.x - o.x) <= 1e-8 * np.linalg.norm(o.x)


def test_dot_fallback_out_of_scaled_range(B):
    """PCG_DOTS_SPLIT32 on a diagonal matrix with entries 1..1e44 and b_j = min(1, d_j^-3/4):
    the residual grows by 6e21 in the first iteration and w_1 by far more, so entries of r_1,
    w_1 leave the binary32 range around the scale taken from gamma_0, delta_0 and those
    threads sum in binary64.  The first scalars still follow the oracle."""
    import math
    n = 64
    d = np.logspace(0, 44, n)
    b = np.minimum(1.0, d ** -0.75)
    P = S.Problem(S.CSR32, row_ptr=np.arange(n + 1, dtype=np.int32), col=np.arange(n, dtype=np.int32), val=d,
                  n_csr=n)
    # precondition, from the oracle's r_1, w_1 and the documented scale rule: some scaled entry
    # reaches 2^56, the FP32-pipe limit
    o1 = oracle.pcg_sh(P, b, sigma=0.0, maxit=1, log_every=0, want_state=True)
    g0 = float(np.dot(b, b))
    d0 = float(np.dot(d * b, b))
    sr = 20 - ((math.frexp(g0)[1] - 1) // 2 + 1)
    sw = sr - math.frexp(abs(d0 / g0))[1]
    assert math.log2(np.abs(o1.state["w"]).max()) + sw >= 56
    g, o = run_both(B, P, b, "pcg", 0.0, 4, flags=B.PCG_DOTS_SPLIT32)
    g64, _ = run_both(B, P, b, "pcg", 0.0, 4)
    assert g.iters == o.iters == 4
    check_scalars(g, o, k=4)
    check_scalars(g64, o, k=4)


def test_random_sdd_csr(B):
    rng = np.random.default_rng(3)
    n = 5000
    rows, cols = [], []
    for i in range(n):
        k = rng.integers(3, 13)
        js = rng.integers(0, n, size=k)
        js = js[js != i]
        rows += [i] * len(js)
        cols += list(js)
    import scipy.sparse as sp
    U = sp.coo_matrix((-rng.random(len(rows)), (rows, cols)), shape=(n, n)).tocsr()
    A = (U + U.T).tocsr()
    A.sum_duplicates()
    d = np.asarray(np.abs(A).sum(axis=1)).ravel() * 1.01 + 1e-3
    A = (A + sp.diags(d)).tocsr()
    A.sort_indices()
    P = S.Problem(S.CSR32, row_ptr=A.indptr.astype(np.int32), col=A.indices.astype(np.int32),
                  val=A.data.astype(np.float64), n_csr=n)
    b = S.normal(9, n)
    g, o = run_both(B, P, b, "spcg", float(np.median(d)) * 0.5, maxit=80)
    check_scalars(g, o)
    check_final(g, o, np.linalg.norm(b))


# ---------------------------------------------------------------- edge cases

def test_single_unknown(B):
    P = S.laplacian_2d(1, 1)            # A = [4]
    b = np.array([3.0])
    with B.Solver(P) as s:
        r = s.solve(b, method="spcg", sigma=1.0, tol=1e-15, maxit=5)
    assert r.status == B.PCG_OK and r.iters == 1
    assert abs(r.x[0] - 0.75) <= 1e-15


def test_zero_rhs_converges_immediately(B):
    P = S.laplacian_3d(8)
    with B.Solver(P) as s:
        r = s.solve(np.zeros(P.n), method="spcg", sigma=6.0, tol=1e-10, maxit=50)
    assert r.status == B.PCG_OK and r.iters == 0 and np.all(r.x == 0)


def test_maxit_zero(B):
    P, b, _ = S.poisson2d_manufactured(16)
    with B.Solver(P) as s:
        r = s.solve(b, method="spcg", sigma=4.0, maxit=0)
    assert r.status == B.PCG_ENOTCONV and r.iters == 0 and np.all(r.x == 0)
    assert abs(r.final_true_relres - 1.0) < 1e-15


def test_nonzero_initial_guess(B):
    P, b, xs = S.poisson2d_manufactured(40)
    x0 = S.uniform_pm1(3, P.n)
    g, o = run_both(B, P, b, "spcg", 4.0, maxit=50, x0=x0)
    check_scalars(g, o)
    np.testing.assert_allclose(g.x, o.x, rtol=1e-9, atol=1e-12)


def test_tolerance_stop_matches_oracle(B):
    P, b, xs = S.poisson2d_manufactured(64)
    g, o = run_both(B, P, b, "spcg", 4.0, maxit=2000, tol=1e-9)
    assert g.status == B.PCG_OK and o.status == 1
    assert abs(g.iters - o.iters) <= 1
    assert g.final_rec_relres <= 1e-9


def test_breakdown_on_indefinite(B):
    """An indefinite matrix gives non-positive curvature: the solve stops with EBREAKDOWN."""
    n = 64
    d = np.ones(n)
    d[::2] = -1.0
    P = S.Problem(S.CSR32, row_ptr=np.arange(n + 1, dtype=np.int32), col=np.arange(n, dtype=np.int32),
                  val=d, n_csr=n)
    b = np.ones(n)
    with B.Solver(P) as s:
        r = s.solve(b, method="spcg", sigma=0.5, maxit=10)
        c = s.solve(b, method="cg", maxit=10)
    assert r.status == B.PCG_EBREAKDOWN
    assert c.status == B.PCG_EBREAKDOWN
    o = oracle.pcg_sh(P, b, sigma=0.5, maxit=10)
    assert o.status == 2 and o.iters == r.iters


def test_invalid_arguments(B):
    P, b, _ = S.poisson2d_manufactured(8)
    from paper_1706_05988_gb300 import pcg as C
    with B.Solver(P) as s:
        x = np.empty(P.n)
        assert C.pcg_solve(s.ctx, b, None, 2, -1.0, 0.0, 5, 0, x, None) == C.PCG_EINVAL       # sigma < 0
        assert C.pcg_solve(s.ctx, b, None, 2, float("nan"), 0.0, 5, 0, x, None) == C.PCG_EINVAL
        assert C.pcg_solve(s.ctx, b, None, 9, 0.0, 0.0, 5, 0, x, None) == C.PCG_EINVAL
        assert C.pcg_solve(s.ctx, b, None, 2, 0.0, -1.0, 5, 0, x, None) == C.PCG_EINVAL
        assert C.pcg_solve(s.ctx, b, None, 2, 0.0, 0.0, -1, 0, x, None) == C.PCG_EINVAL
        assert C.pcg_solve(s.ctx, b, None, 2, 0.0, 0.0, 5, 7, x, None) == C.PCG_EINVAL        # precision
        assert C.pcg_solve(s.ctx, b, None, 0, 0.0, 0.0, 5, 1, x, None) == C.PCG_ENOTIMPL      # mixed CG
        # the context stays usable after rejected calls
        r = s.solve(b, method="spcg", sigma=4.0, maxit=5)
        assert r.iters == 5


# ---------------------------------------------------------------- properties of the GPU path itself

def test_deterministic_and_pcg_is_sigma0(B):
    P, b, _ = S.poisson3d_manufactured(32)
    with B.Solver(P) as s:
        a = s.solve(b, method="spcg", sigma=0.0, maxit=100)
        a2 = s.solve(b, method="spcg", sigma=0.0, maxit=100)
        p = s.solve(b, method="pcg", sigma=3.0, maxit=100)      # sigma ignored by p-CG
    assert np.array_equal(a.x, a2.x) and np.array_equal(a.alpha, a2.alpha)
    assert np.array_equal(a.x, p.x) and np.array_equal(a.rec, p.rec)


def test_graph_replay_matches_direct_launches(B):
    """Without profiling and true-residual logging, the iteration launches are replayed from
    a CUDA graph of 32; with logging (here never due) they are launched one by one.  The
    kernel is the same, so iterates, histories and stop iteration are bit-identical, for a
    fixed count (graphs plus a ragged remainder) and for a tolerance stop (polled chunks)."""
    P, b, _ = S.poisson2d_manufactured(100)
    with B.Solver(P) as s:
        for tol, maxit in ((0.0, 203), (1e-9, 5000)):
            g = s.solve(b, method="spcg", sigma=4.0, tol=tol, maxit=maxit, true_every=0)
            d = s.solve(b, method="spcg", sigma=4.0, tol=tol, maxit=maxit, true_every=maxit + 1)
            assert g.iters == d.iters and g.status == d.status
            assert np.array_equal(g.x, d.x)
            k = g.iters + 1
            assert np.array_equal(g.alpha[:k], d.alpha[:k]) and np.array_equal(g.rec[:k], d.rec[:k])
        assert g.iters < 5000
        # a second context on the same problem rebuilds nothing of the first one's graph
        with B.Solver(P) as s2:
            g2 = s2.solve(b, method="spcg", sigma=4.0, tol=0.0, maxit=203, true_every=0)
        g3 = s.solve(b, method="spcg", sigma=4.0, tol=0.0, maxit=203, true_every=0)
        assert np.array_equal(g2.x, g3.x)


def test_device_entry_point_matches_host(B):
    import torch
    P, b, _ = S.poisson3d_manufactured(24)
    with B.Solver(P) as s:
        h = s.solve(b, method="spcg", sigma=6.0, maxit=40)
        db = torch.from_numpy(b).cuda()
        d = s.solve(db, method="spcg", sigma=6.0, maxit=40, device=True)
        # a misaligned device b (offset by one element) is copied internally
        buf = torch.empty(P.n + 1, dtype=torch.float64, device="cuda")
        buf[1:] = db
        d2 = s.solve(buf[1:], method="spcg", sigma=6.0, maxit=40, device=True)
    assert np.array_equal(h.x, d.x.cpu().numpy())
    assert np.array_equal(h.x, d2.x.cpu().numpy())


def test_device_matrix_pointers(B):
    import torch
    P = S.varcoef_3d(16, block=4, seed=8)
    dev = {k: torch.from_numpy(getattr(P, k)).cuda() for k in ("diag", "ax", "ay", "az")}
    b = S.normal(4, P.n)
    with B.Solver(P) as s1, B.Solver(P, device_arrays=dev) as s2:
        r1 = s1.solve(b, method="spcg", sigma=1.0, maxit=30)
        r2 = s2.solve(b, method="spcg", sigma=1.0, maxit=30)
    assert np.array_equal(r1.x, r2.x)


# ---------------------------------------------------------------- shift selection

def test_psi_matches_oracle(B):
    from oracle import psi as PS
    P, b = S.lapl200()
    o = oracle.pcg_sh(P, b, sigma=4.0, maxit=301, log_every=0)
    grid = np.array([0.0, 1.0, 2.0, 4.0, 6.0, 7.5, 9.0])
    with B.Solver(P) as s:
        from paper_1706_05988_gb300 import pcg as C
        g = C.pcg_psi(s.ctx, o.alpha, o.beta, 300, grid)
    ref = np.array([PS.psi(o.alpha, o.beta, 300, sg) for sg in grid])
    fin = np.isfinite(ref) & (ref < 1e100)
    assert rel(g[fin], ref[fin]) < 1e-9
    assert np.all(g[~fin] > 1e100)


def test_select_sigma_lapl200(B):
    P, b = S.lapl200()
    with B.Solver(P) as s:
        from paper_1706_05988_gb300 import pcg as C
        sg, psi = C.pcg_select_sigma(s.ctx, b, 300, np.linspace(0.5, 8.0, 16))
    assert sg == 4.0


def test_select_sigma_lapl3d_matches_oracle(B):
    """The second selection case (32^3 Laplacian, 100-iteration unshifted pilot): the device's
    pilot and psi evaluation pick the oracle's shift, with psi on the grid to 1e-6."""
    from oracle import psi as PS
    from paper_1706_05988_gb300 import pcg as C
    P, b, _ = S.poisson3d_manufactured(32)
    grid = np.linspace(0.5, 12.0, 24)
    pil = oracle.pcg_sh(P, b, sigma=0.0, maxit=100, log_every=0)
    so, vo = PS.select_sigma(pil.alpha, pil.beta, 99, grid)
    with B.Solver(P) as s:
        sg, psi = C.pcg_select_sigma(s.ctx, b, 100, grid)
    assert sg == so == 1.0
    assert rel(psi, vo) < 1e-6


# ---------------------------------------------------------------- full size: 256^3 stencil (n = 16.8M)

@pytest.fixture(scope="module")
def big():
    P, b, xs = S.poisson3d_manufactured(256)
    return P, b


def full_size_x_check(gx, ox):
    """Every entry of the iterate after 20 iterations: the two sides differ only by
    summation order, so each entry agrees to a few units of 1e-12 of the iterate's scale."""
    scale = np.abs(ox).max()
    err = np.abs(gx - ox)
    assert np.all(err <= 1e-10 * np.abs(ox) + 1e-12 * scale), float(np.max(err / (np.abs(ox) + scale)))


def test_full_size_first_iterations_vs_oracle(B, big):
    """Same launch configuration as the benchmark (256^3, sigma = 6): alpha_i, beta_i of the
    first 20 iterations at 1e-10 and all 16.8M entries of x_20 against the oracle."""
    P, b = big
    with B.Solver(P) as s:
        g = s.solve(b, method="spcg", sigma=6.0, maxit=N_SCALARS, true_every=0)
    o = oracle.pcg_sh(P, b, sigma=6.0, maxit=N_SCALARS, log_every=0)
    assert g.iters == o.iters == N_SCALARS
    check_scalars(g, o, k=N_SCALARS)
    full_size_x_check(g.x, o.x)


def test_full_size_1000_iterations_properties(B, big):
    """1,000 iterations at 256^3: the residual falls steadily and the gap stays at rounding level."""
    P, b = big
    with B.Solver(P) as s:
        g = s.solve(b, method="spcg", sigma=6.0, maxit=1000, true_every=250)
    assert g.iters == 1000
    assert np.all(np.diff(g.rec[::50]) < 0)
    assert g.final_true_relres < 1e-3
    bn = np.linalg.norm(b)
    assert np.nanmax(g.gap) / bn < 1e-12
    assert abs(g.final_true_relres - g.final_rec_relres) < 1e-10


def test_full_size_csr_first_iterations_vs_oracle(B, big):
    """The same 256^3 Laplacian assembled as CSR with int32 indices (117,047,296 entries, the
    benchmark's CSR form): the first 20 iterations and every entry of x_20 against the oracle
    on the same CSR arrays."""
    P, b = big
    Pc = S.to_csr(P)
    assert Pc.nnz == 117_047_296
    with B.Solver(Pc) as s:
        g = s.solve(b, method="spcg", sigma=6.0, maxit=N_SCALARS, true_every=0)
    o = oracle.pcg_sh(Pc, b, sigma=6.0, maxit=N_SCALARS, log_every=0)
    assert g.iters == o.iters == N_SCALARS
    check_scalars(g, o, k=N_SCALARS)
    full_size_x_check(g.x, o.x)


@pytest.mark.parametrize("method,sigma", [("cg", 0.0), ("spcg", 4.0)])
def test_true_residual_stop(B, method, sigma):
    """The 100x100 Poisson run of the accuracy study: at most 2,000 iterations or a true relative
    residual of 1e-14, checked every iteration (PCG_PARAM_TRUE_TOL); the stop iteration and the
    final residual follow the oracle's true-residual stop."""
    from paper_1706_05988_gb300 import pcg as C
    P, b, _ = S.poisson2d_manufactured(100)
    with B.Solver(P) as s:
        assert C.pcg_set_param(s.ctx, C.PCG_PARAM_TRUE_TOL, 1e-14) == C.PCG_OK
        g = s.solve(b, method=method, sigma=sigma, maxit=2000, true_every=1)
        assert C.pcg_set_param(s.ctx, C.PCG_PARAM_TRUE_TOL, -1.0) == C.PCG_EINVAL
    if method == "cg":
        o = oracle.cg(P, b, maxit=2000, ttol=1e-14, log_every=1)
    else:
        o = oracle.pcg_sh(P, b, sigma=sigma, maxit=2000, ttol=1e-14, log_every=1)
    bn = np.linalg.norm(b)
    assert o.status == 1 and g.status == B.PCG_OK, (o.status, g.status)
    assert abs(g.iters - o.iters) <= 2, (g.iters, o.iters)
    assert g.final_true_relres <= 1e-14 and o.true[-1] / bn <= 1e-14


# ---------------------------------------------------------------- staged (TMA) sweep

STAGE_SHAPES = [("3d_even", lambda: S.laplacian_3d(20, 18, 16)), ("3d_cube64", lambda: S.laplacian_3d(64)),
                ("3d_ragged_chunk", lambda: S.laplacian_3d(34, 30, 7)), ("2d_even", lambda: S.laplacian_2d(64, 45)),
                ("3d_fp64rows", lambda: S.laplacian_3d(24, 22, 10))]


@pytest.mark.parametrize("name,maker", STAGE_SHAPES, ids=[s[0] for s in STAGE_SHAPES])
@pytest.mark.parametrize("stages", [2, 3])
def test_staged_sweep_vs_oracle_and_register_sweep(B, name, maker, stages):
    """The fused iteration with every operand staged by TMA bulk copies (a ring of 2 or 3
    chunks) against the oracle (parity bar) and against the register sweep: the same
    arithmetic on the same units, so bit for bit where both sweeps have the same grid (the
    small shapes), and to 1e-12 where the staged sweep's smaller resident grid (3 or 2 blocks
    per SM instead of 4) changes the order of the block partials (64^3: 512 blocks needed).
    The shapes cover chunks that cross rows and planes, a last chunk shorter than the others
    (34*30*7 = 7,140 unknowns = 13 chunks of 512 and 484 more), the 2D stencil and the
    binary64 row sums."""
    from paper_1706_05988_gb300 import pcg as C
    P = maker()
    b = S.normal(11, P.n)
    flags = B.PCG_STENCIL_FP64_SUM if name == "3d_fp64rows" else 0
    sigma = shift_for(P)
    with B.Solver(P, flags=flags) as s:
        assert C.pcg_set_param(s.ctx, C.PCG_PARAM_ITER_STAGES, float(stages)) == C.PCG_OK
        assert C.pcg_get_param(s.ctx, C.PCG_PARAM_ITER_STAGES) == stages
        gs = s.solve(b, method="spcg", sigma=sigma, maxit=30, true_every=1)
        assert C.pcg_set_param(s.ctx, C.PCG_PARAM_ITER_STAGES, 0.0) == C.PCG_OK
        assert C.pcg_get_param(s.ctx, C.PCG_PARAM_ITER_STAGES) == 0
        g0 = s.solve(b, method="spcg", sigma=sigma, maxit=30, true_every=1)
    o = oracle.pcg_sh(P, b, sigma=sigma, maxit=30, log_every=1)
    check_scalars(gs, o)
    check_final(gs, o, np.linalg.norm(b))
    if P.n // 512 < 2 * 152:       # both grids are the blocks the problem needs
        assert np.array_equal(gs.x, g0.x) and np.array_equal(gs.alpha, g0.alpha)
        assert np.array_equal(gs.beta, g0.beta)
    else:
        assert rel(gs.alpha, g0.alpha) <= 1e-12 and rel(gs.beta[1:], g0.beta[1:]) <= 1e-12
        assert np.linalg.norm(gs.x - g0.x) <= 1e-12 * np.linalg.norm(g0.x)


def test_staged_sweep_where_it_applies(B):
    """The register sweep is the default; asked for, the staged sweep is taken on
    constant-coefficient stencils with an even row length (the 256^3 workload among them),
    while CSR, variable coefficients and odd rows stay on the register sweep."""
    from paper_1706_05988_gb300 import pcg as C
    for P, want in ((S.laplacian_3d(256), 2), (S.laplacian_2d(100, 100), 2), (S.laplacian_3d(15, 17, 9), 0),
                    (S.varcoef_3d(24, block=8, seed=3), 0), (S.to_csr(S.laplacian_3d(18, 14, 10)), 0)):
        with B.Solver(P) as s:
            assert C.pcg_get_param(s.ctx, C.PCG_PARAM_ITER_STAGES) == 0
            assert C.pcg_set_param(s.ctx, C.PCG_PARAM_ITER_STAGES, 2.0) == C.PCG_OK
            assert C.pcg_get_param(s.ctx, C.PCG_PARAM_ITER_STAGES) == want, (P.n, want)
            assert C.pcg_set_param(s.ctx, C.PCG_PARAM_ITER_STAGES, 1.0) == C.PCG_EINVAL

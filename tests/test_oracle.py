"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test states what fixes the expected value: a published value of the
paper, a closed form, a library routine, exact rational arithmetic, or an
invariant of the method.
"""
import json
import os
from fractions import Fraction as F

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp

import oracle
import synthetic as S
from oracle import exact as EX
from oracle import psi as PS

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_csr(A):
    """Dense -> synthetic CSR problem (all structural entries kept)."""
    A = np.asarray(A, dtype=np.float64)
    m = sp.csr_matrix(A)
    m.sort_indices()
    return S.Problem(S.CSR32, row_ptr=m.indptr.astype(np.int32), col=m.indices.astype(np.int32),
                     val=m.data.astype(np.float64), n_csr=A.shape[0])


def scipy_of(P):
    c = S.to_csr(P)
    return sp.csr_matrix((c.val, c.col, c.row_ptr), shape=(c.n, c.n))


def spd_int(n, seed):
    """Small SPD integer matrix B^T B + n I (exact in rationals and in binary64)."""
    rng = np.random.default_rng(seed)
    B = rng.integers(-3, 4, size=(n, n))
    return (B.T @ B + n * np.eye(n, dtype=np.int64)).astype(np.int64)


# ---------------------------------------------------------------- generators

def test_splitmix64_published_values():
    # SplitMix64 reference outputs for seed 0 (Steele/Lea/Flood; Vigna's splitmix64.c)
    v = S.splitmix64(0, 3)
    assert [int(x) for x in v] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_dyadic_inputs_in_range():
    x = S.dyadic_uniform_pm1(0, 100000)
    assert x.min() >= -1.0 and x.max() < 1.0
    assert np.all(x * 2 ** 30 == np.round(x * 2 ** 30))
    assert abs(x.mean()) < 0.01 and abs(x.var() - 1 / 3) < 0.01


# ---------------------------------------------------------------- operator

@pytest.mark.parametrize("maker", [
    lambda: S.laplacian_2d(7, 5),
    lambda: S.laplacian_3d(5, 4, 3),
    lambda: S.varcoef_2d(6, 5, seed=3),
    lambda: S.varcoef_3d(6, block=2, seed=4),
])
def test_operator_matches_scipy(maker):
    """Matrix-free stencil of the oracle vs the generator's CSR assembly multiplied by scipy."""
    P = maker()
    x = S.uniform_pm1(11, P.n)
    y = oracle.apply(P, x)
    ref = scipy_of(P) @ x
    np.testing.assert_allclose(y, ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max())
    # and the oracle's CSR path on the same matrix
    y2 = oracle.apply(S.to_csr(P), x)
    np.testing.assert_allclose(y2, ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max())


def test_laplacian_definition_tiny():
    """Row sums / symmetry of the 3D Laplacian from its definition: 6 on the diagonal,
    -1 per interior neighbour, so A*1 = number of boundary faces of each cell."""
    P = S.laplacian_3d(4, 3, 5)
    y = oracle.apply(P, np.ones(P.n)).reshape(5, 3, 4)
    k, j, i = np.meshgrid(range(5), range(3), range(4), indexing="ij")
    faces = sum((c).astype(int) for c in (i == 0, i == 3, j == 0, j == 2, k == 0, k == 4))
    assert np.array_equal(y, faces.astype(float))
    M = scipy_of(P).toarray()
    assert np.array_equal(M, M.T) and np.all(np.linalg.eigvalsh(M) > 0)


def test_rhs_exact():
    P, b, xs = S.poisson3d_manufactured(9)
    assert np.array_equal(oracle.apply(P, xs), b)
    P2, b2, xs2 = S.poisson2d_manufactured(13)
    assert np.array_equal(oracle.apply(P2, xs2), b2)


def test_varcoef_is_spd_and_contrast():
    P = S.varcoef_3d(16, block=8, seed=0)
    M = scipy_of(P).toarray()
    assert np.allclose(M, M.T)
    ev = np.linalg.eigvalsh(M)
    assert ev.min() > 0
    k = P.meta["kappa"]
    assert k.min() >= 1e-3 and k.max() <= 1e3


# ---------------------------------------------------------------- classic CG

@pytest.mark.parametrize("n", [8, 24, 64])
def test_cg_matches_cholesky(n):
    A = spd_int(n, n)
    b = S.uniform_pm1(n, n)
    ref = scipy.linalg.cho_solve(scipy.linalg.cho_factor(A.astype(float)), b)
    r = oracle.cg(dense_csr(A), b, maxit=3 * n, rtol=1e-15)
    np.testing.assert_allclose(r.x, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_cg_finite_termination_distinct_eigenvalues():
    """Diagonal A with k distinct eigenvalues: CG's residual vanishes after k steps."""
    lam = np.array([1.0, 2.0, 5.0, 7.0, 11.0])
    d = np.repeat(lam, 10)
    A = np.diag(d)
    b = S.uniform_pm1(3, d.size)
    r = oracle.cg(dense_csr(A), b, maxit=len(lam))
    assert r.true[-1] <= 1e-13 * np.linalg.norm(b)
    assert r.true[len(lam) - 1] > 1e-6           # and not one step earlier


def test_cg_scaled_identity_one_step():
    c = 4.0
    A = c * np.eye(12)
    b = S.uniform_pm1(5, 12)
    r = oracle.cg(dense_csr(A), b, maxit=3, rtol=1e-16)
    assert r.alpha[0] == 1.0 / c
    assert np.array_equal(r.x, b / c)
    assert r.iters == 1


# ---------------------------------------------------------------- exact arithmetic

@pytest.mark.parametrize("n,seed", [(6, 1), (9, 2)])
def test_exact_cg_terminates_at_solution(n, seed):
    import sympy
    A = spd_int(n, seed)
    b = [F(int(v)) for v in np.random.default_rng(seed).integers(-5, 6, n)]
    Af = [[F(int(v)) for v in row] for row in A]
    _, _, x, _ = EX.cg(Af, b, iters=n)
    xs = sympy.Matrix(A.tolist()).LUsolve(sympy.Matrix([int(v) for v in b]))
    assert [sympy.Rational(v.numerator, v.denominator) for v in x] == list(xs)


@pytest.mark.parametrize("sigma", [F(0), F(1, 2), F(4), F(7, 3)])
@pytest.mark.parametrize("precond", [False, True])
def test_exact_pcg_sh_equals_cg(sigma, precond):
    """Algorithms 1 and 3 coincide in exact arithmetic for every shift (Section 3)."""
    n = 7
    A = spd_int(n, 5)
    Af = [[F(int(v)) for v in row] for row in A]
    b = [F(int(v)) for v in np.random.default_rng(9).integers(-5, 6, n)]
    minv = [F(1, int(A[i, i])) for i in range(n)] if precond else None
    a1, b1, x1, xs1 = EX.cg(Af, b, iters=n, minv=minv)
    a3, b3, x3, xs3 = EX.pcg_sh(Af, b, sigma=sigma, iters=n, minv=minv)
    assert a1 == a3 and b1 == b3 and xs1 == xs3


@pytest.mark.parametrize("sigma", [0.0, 0.5, 4.0])
@pytest.mark.parametrize("precond", [False, True])
def test_fp64_oracle_matches_exact(sigma, precond):
    """The C oracle's alpha_i, beta_i, x_i agree with exact rational CG to rounding level."""
    n = 10
    A = spd_int(n, 17)
    rng = np.random.default_rng(4)
    bi = rng.integers(-9, 10, n)
    Af = [[F(int(v)) for v in row] for row in A]
    minv_f = [F(1, int(A[i, i])) for i in range(n)] if precond else None
    minv = np.array([1.0 / A[i, i] for i in range(n)]) if precond else None
    a_ex, b_ex, _, xs_ex = EX.cg(Af, [F(int(v)) for v in bi], iters=n, minv=minv_f)
    k = len(a_ex) - 1
    runs = [oracle.cg(dense_csr(A), bi.astype(float), maxit=k, minv=minv),
            oracle.pcg_sh(dense_csr(A), bi.astype(float), sigma=sigma, maxit=k, minv=minv)]
    ea = np.array([float(v) for v in a_ex[:k]])
    eb = np.array([float(v) for v in b_ex[:k]])
    for r in runs:
        assert r.iters == k
        # first half: rounding level; all iterations: far below any transcription error (O(1))
        np.testing.assert_allclose(r.alpha[:5], ea[:5], rtol=1e-12)
        np.testing.assert_allclose(r.beta[1:5], eb[1:5], rtol=1e-12)
        np.testing.assert_allclose(r.alpha, ea, rtol=1e-7)
        np.testing.assert_allclose(r.beta[1:], eb[1:], rtol=1e-7)
        np.testing.assert_allclose(r.x, [float(v) for v in xs_ex[k]], rtol=1e-7, atol=1e-12)


# ---------------------------------------------------------------- invariants of Algorithm 3

def test_pcg_sigma0_is_algorithm2_bitwise():
    """Algorithm 3 with sigma = 0 reverts to Algorithm 2 (end of Section 2.2)."""
    P, b, _ = S.poisson2d_manufactured(30)
    r3 = oracle.pcg_sh(P, b, sigma=0.0, maxit=120)
    r2 = oracle.pcg(P, b, maxit=120)
    assert np.array_equal(r3.alpha, r2.alpha) and np.array_equal(r3.beta, r2.beta)
    assert np.array_equal(r3.x, r2.x) and np.array_equal(r3.rec, r2.rec)


def test_identity_preconditioner_aliases():
    """With M = I: u = r, q = s, t = p and m = w hold bit for bit."""
    P, b, _ = S.poisson2d_manufactured(20)
    r = oracle.pcg_sh(P, b, sigma=4.0, maxit=37, want_state=True)
    st = r.state
    assert np.array_equal(st["u"], st["r"]) and np.array_equal(st["q"], st["s"])
    assert np.array_equal(st["t"], st["p"])


@pytest.mark.parametrize("k", [1, 5, 20])
@pytest.mark.parametrize("precond", [False, True])
def test_auxiliary_definitions_hold(k, precond):
    """Recursive w, s, z, r, u, q match their definitions (Eq. pipe_cg_shift_aux) early on."""
    P = S.varcoef_2d(24, 20, seed=2) if precond else S.laplacian_2d(24, 20)
    sigma = 1.0 if precond else 3.0          # inside the spectrum of A M^-1 (a too large shift destabilises)
    b = S.normal(1, P.n)
    minv = 1.0 / scipy_of(P).diagonal() if precond else None
    st = oracle.pcg_sh(P, b, sigma=sigma, maxit=k, minv=minv, want_state=True).state
    Mi = (lambda v: v) if minv is None else (lambda v: minv * v)
    A = lambda v: oracle.apply(P, v)

    def rel(a, b_):
        return np.linalg.norm(a - b_) / max(np.linalg.norm(b_), 1e-300)

    tol = 1e-11
    assert rel(A(st["u"]) - sigma * st["r"], st["w"]) < tol        # w = A u - sigma r
    assert rel(A(st["p"]) - sigma * st["t"], st["s"]) < tol        # s = A p - sigma t
    assert rel(A(st["q"]), st["z"]) < tol                          # z = A q
    assert rel(Mi(st["r"]), st["u"]) < tol                         # u = M^-1 r
    assert rel(Mi(st["s"]), st["q"]) < tol                         # q = M^-1 s
    assert rel(Mi(st["t"]), st["p"]) < tol                         # p = M^-1 t
    assert rel(b - A(st["x"]), st["r"]) < 1e-10                    # r = b - A x


# ---------------------------------------------------------------- Table 1, lapl200

@pytest.fixture(scope="module")
def lapl200_runs():
    P, b = S.lapl200()
    return {
        "cg": oracle.cg(P, b, maxit=500, log_every=10),
        "pcg": oracle.pcg_sh(P, b, sigma=0.0, maxit=500, log_every=10),
        "pcgsh": oracle.pcg_sh(P, b, sigma=4.0, maxit=500, log_every=10),
    }


def test_lapl200_table1(lapl200_runs):
    g = json.load(open(os.path.join(GOLDEN, "lapl200_table1.json")))
    cg, pcg, sh = lapl200_runs["cg"], lapl200_runs["pcg"], lapl200_runs["pcgsh"]
    assert abs(cg.rec[0] - g["r0_norm"]) < 1e-12
    assert cg.iters == 500 and sh.iters == 500
    lo, hi = g["true_residual"]["cg"] / 2.3, g["true_residual"]["cg"] * 2.1
    assert lo <= cg.true[-1] <= hi
    assert lo <= sh.true[-1] <= hi
    # p-CG loses attainable accuracy: its last logged true residual sits >= 100x above CG's
    last = pcg.true[~np.isnan(pcg.true)][-1]
    assert last >= 100 * cg.true[-1]


def test_lapl200_gaps(lapl200_runs):
    """CG's residual gap is only accumulated (P = 1, Eq. gap_f0_cg); p-CG's is amplified."""
    cg, pcg, sh = lapl200_runs["cg"], lapl200_runs["pcg"], lapl200_runs["pcgsh"]
    gcg = np.nanmax(cg.gap)
    assert gcg < 2e-11
    assert np.nanmax(pcg.gap) > 100 * gcg
    assert np.nanmax(sh.gap) < 5 * gcg


def test_psi_lapl200(lapl200_runs):
    """psi_500(sigma*=4) = 3.46e2 for lapl200 (Section 5.1); the unshifted value is orders larger."""
    g = json.load(open(os.path.join(GOLDEN, "lapl200_table1.json")))
    sh = lapl200_runs["pcgsh"]
    P, b = S.lapl200()
    sh501 = oracle.pcg_sh(P, b, sigma=4.0, maxit=501, log_every=0)
    v = PS.psi(sh501.alpha, sh501.beta, g["iterations"], g["sigma_star"])
    assert abs(v / g["psi"]["sigma_star"] - 1) < 0.01
    pcg = lapl200_runs["pcg"]
    i = min(pcg.iters - 1, 500)
    v0 = PS.psi(pcg.alpha, pcg.beta, i, 0.0)
    assert v0 > 1e4 * v
    assert sh.iters == 500


def test_psi_closed_form_one_step():
    """psi_1 with beta = 0, alpha*sigma = 1: P = [[1,0,-c,0],[0,0,1,0],0,0] with c = alpha,
    whose largest singular value is sqrt(((2+c^2)+sqrt((2+c^2)^2-4))/2)."""
    c, sigma = 0.3, 1 / 0.3
    al, be = np.array([0.0, c]), np.array([0.0, 0.0])
    e = 2 + c * c
    assert abs(PS.psi(al, be, 1, sigma) - np.sqrt((e + np.sqrt(e * e - 4)) / 2)) < 1e-14


def test_psi_varsh_closed_form_one_step():
    """Variable shift, one step, beta = 0, alpha*sigma_0 = 1 (sigma_0 = sigma_{i-1}): the nonzero part of
    P is [[1, -c], [0, 1], [0, -d]] in rows 0, 1, 3 and columns 0, 2 (d = sigma_1 - sigma_0), whose
    largest singular value is sqrt((t + sqrt(t^2 - 4 det)) / 2), t = 2 + c^2 + d^2, det = 1 + d^2."""
    c, s0, d = 0.3, 1 / 0.3, 0.7
    al, be = np.array([0.0, c]), np.array([0.0, 0.0])
    t, det = 2 + c * c + d * d, 1 + d * d
    want = np.sqrt((t + np.sqrt(t * t - 4 * det)) / 2)
    assert abs(PS.psi_varsh(al, be, 1, [0.0, s0, s0 + d]) - want) < 1e-14
    # the change of shift is what couples the j-gap in: with d = 0 it is the constant-shift value
    e = 2 + c * c
    assert abs(PS.psi_varsh(al, be, 1, [0.0, s0, s0]) - np.sqrt((e + np.sqrt(e * e - 4)) / 2)) < 1e-14


def test_psi_varsh_constant_schedule_is_psi(lapl200_runs):
    """A constant schedule gives psi_i(sigma) of Eq. (functionpsi) on a real alpha/beta history
    (lapl200's unshifted pilot run, pinned to the paper's 3.46e2 at sigma = 4 above)."""
    pcg = lapl200_runs["pcg"]
    for sigma in (0.0, 2.5, 4.0):
        sh = np.full(202, sigma)
        assert abs(PS.psi_varsh(pcg.alpha, pcg.beta, 200, sh) / PS.psi(pcg.alpha, pcg.beta, 200, sigma) - 1) < 1e-12


def test_psi_product_order_matters():
    """psi uses P_i ... P_j (newest on the left); the reversed product gives another value,
    so the lapl200 pin above also fixes the order."""
    P, b = S.lapl200()
    r = oracle.pcg_sh(P, b, sigma=4.0, maxit=201, log_every=0)
    good = PS.psi(r.alpha, r.beta, 200, 4.0)
    Q, best = np.eye(4), 0.0
    for j in range(200, 0, -1):
        Q = PS.prop_matrix(r.alpha[j], r.beta[j], 4.0) @ Q
        best = max(best, np.linalg.norm(Q, 2))
    assert abs(best / good - 1) > 0.01


def test_select_sigma_lapl200(lapl200_runs):
    """The a-posteriori shift from the coefficient history of an unshifted p-CG pilot run
    (Section 5.1; 300 iterations, before that run breaks down near 450) reproduces Table 1's
    sigma* = 4.00, and so does the p-CG-sh(4) history of 500 iterations."""
    P, b = S.lapl200()
    pil = oracle.pcg_sh(P, b, sigma=0.0, maxit=300, log_every=0)
    grid = np.linspace(0.5, 8.0, 16)
    s, vals = PS.select_sigma(pil.alpha, pil.beta, 299, grid)
    assert s == 4.0
    assert vals[0] > 5 * vals.min()
    # beyond the top of the spectrum (lambda_max < 8) psi explodes: the cliff the rule avoids
    assert PS.psi(pil.alpha, pil.beta, 299, 9.0) > 1e6 * vals.min()
    sh = lapl200_runs["pcgsh"]
    assert PS.select_sigma(sh.alpha, sh.beta, 499, grid)[0] == 4.0


def test_select_sigma_second_case_lapl3d():
    """A second case for the selection rule: the 32^3 Laplacian with a manufactured solution.
    The shift chosen from a 100-iteration unshifted pilot brings p-CG-sh to CG's attainable
    accuracy, while unshifted p-CG stalls at least 100 times above it (Table 1's pattern)."""
    P, b, _ = S.poisson3d_manufactured(32)
    bn = np.linalg.norm(b)
    pil = oracle.pcg_sh(P, b, sigma=0.0, maxit=100, log_every=0)
    s, vals = PS.select_sigma(pil.alpha, pil.beta, 99, np.linspace(0.5, 12.0, 24))
    assert 0.5 <= s <= 6.0
    cg = oracle.cg(P, b, maxit=1500, log_every=100)
    p0 = oracle.pcg_sh(P, b, sigma=0.0, maxit=1500, log_every=100)
    ps = oracle.pcg_sh(P, b, sigma=s, maxit=1500, log_every=100)
    assert ps.true[-1] / bn <= 10 * cg.true[-1] / bn
    assert np.nanmin(p0.true) / bn >= 100 * cg.true[-1] / bn


# ---------------------------------------------------------------- Algorithm 4 (variable shift)

@pytest.mark.parametrize("precond", [False, True])
def test_exact_varsh_equals_cg(precond):
    """Algorithm 4 coincides with Algorithm 1 in exact arithmetic for any shift sequence (Section 4.1)."""
    n = 7
    A = spd_int(n, 5)
    Af = [[F(int(v)) for v in row] for row in A]
    b = [F(int(v)) for v in np.random.default_rng(9).integers(-5, 6, n)]
    minv = [F(1, int(A[i, i])) for i in range(n)] if precond else None
    shifts = [F(3), F(1, 2), F(4), F(0), F(7, 3), F(5), F(2), F(1), F(6)]
    a1, b1, _, xs1 = EX.cg(Af, b, iters=n, minv=minv)
    a4, b4, _, xs4 = EX.pcg_varsh(Af, b, shifts, iters=n, minv=minv)
    assert a1 == a4 and b1 == b4 and xs1 == xs4


def test_exact_varsh_constant_and_switching_shift():
    """Exact arithmetic: Algorithm 4 with a constant shift equals Algorithm 3 and CG, and a
    shift that switches mid-run (the correction terms then act) still equals CG."""
    n = 6
    A = spd_int(n, 3)
    Af = [[F(int(v)) for v in row] for row in A]
    b = [F(int(v)) for v in np.random.default_rng(2).integers(-5, 6, n)]
    a1, _, _, _ = EX.cg(Af, b, iters=n)
    a3, _, _, _ = EX.pcg_sh(Af, b, sigma=F(2), iters=n)
    a4, _, _, _ = EX.pcg_varsh(Af, b, [F(2)] * (n + 1), iters=n)
    assert a1 == a3 == a4
    a4v, _, _, _ = EX.pcg_varsh(Af, b, [F(2), F(2), F(5)] + [F(5)] * n, iters=n)
    assert a4v == a1


@pytest.mark.parametrize("precond", [False, True])
def test_fp64_varsh_matches_exact(precond):
    n = 10
    A = spd_int(n, 17)
    bi = np.random.default_rng(4).integers(-9, 10, n)
    Af = [[F(int(v)) for v in row] for row in A]
    minv_f = [F(1, int(A[i, i])) for i in range(n)] if precond else None
    minv = np.array([1.0 / A[i, i] for i in range(n)]) if precond else None
    shifts = [0.5, 1.0, 2.0, 1.5, 3.0, 0.25, 1.0, 2.0, 4.0, 1.0, 0.5, 2.0]
    a_ex, b_ex, _, xs_ex = EX.pcg_varsh(Af, [F(int(v)) for v in bi], [F(v) for v in shifts], iters=n, minv=minv_f)
    k = min(len(a_ex) - 1, 6)
    r = oracle.pcg_varsh(dense_csr(A), bi.astype(float), shifts, maxit=k, minv=minv)
    np.testing.assert_allclose(r.alpha, [float(v) for v in a_ex[:k]], rtol=1e-10)
    np.testing.assert_allclose(r.beta[1:], [float(v) for v in b_ex[1:k]], rtol=1e-10)
    np.testing.assert_allclose(r.x, [float(v) for v in xs_ex[k]], rtol=1e-9, atol=1e-12)


def test_varsh_constant_shift_is_algorithm3_bitwise():
    """With sigma_i constant every correction term is an exact zero: Algorithm 4 reproduces
    Algorithm 3 bit for bit."""
    P, b, _ = S.poisson2d_manufactured(30)
    r3 = oracle.pcg_sh(P, b, sigma=4.0, maxit=80)
    r4 = oracle.pcg_varsh(P, b, [4.0] * 81, maxit=80)
    assert np.array_equal(r3.alpha, r4.alpha) and np.array_equal(r3.x, r4.x)


# ---------------------------------------------------------------- gaps g, h, j (Section 3.1)

@pytest.mark.parametrize("sigma,precond", [(F(0), False), (F(3, 2), False), (F(4), True)])
def test_exact_gaps_vanish(sigma, precond):
    """In exact arithmetic the recurrences of Algorithm 3 keep every auxiliary vector equal to
    its definition (Eq. (pipe_cg_shift_aux)): the gaps f, g, h, j are exactly zero."""
    n = 6
    A = spd_int(n, 11)
    Af = [[F(int(v)) for v in row] for row in A]
    b = [F(int(v)) for v in np.random.default_rng(12).integers(-4, 5, n)]
    minv = [F(1, int(A[i, i])) for i in range(n)] if precond else None
    log = []
    EX.pcg_sh(Af, b, sigma=sigma, iters=n, minv=minv, gap_log=log)
    assert len(log) >= 3
    for e in log:
        assert e["f"] == 0 and e["g"] == 0 and e["h"] == 0 and e["j"] == 0


def gap_states(sigma, ks=(120, 121, 122)):
    """lapl200 with shift sigma: the exported vectors after iterations ks, and a run of
    ks[-1] iterations with the gaps logged at every iteration."""
    P, b = S.lapl200()
    st = {k: oracle.pcg_sh(P, b, sigma=sigma, maxit=k, log_every=1, want_state=True).state for k in ks}
    run = oracle.pcg_sh(P, b, sigma=sigma, maxit=ks[-1], log_every=1, gaps=True)
    return P, b, [st[k] for k in ks], run


@pytest.fixture(scope="module")
def gaps_sigma0():
    return gap_states(0.0)


@pytest.fixture(scope="module")
def gaps_sigma4():
    return gap_states(4.0)


def test_logged_gaps_match_their_definitions(gaps_sigma0, gaps_sigma4):
    """||g||, ||h||, ||j|| as logged by the oracle against the definitions recomputed with a
    scipy operator from the exported vectors (iteration 121's p, t, s, q, z; the final u, r,
    w).  Unshifted p-CG has amplified g and h far above rounding (agreement to 1e-5); the
    other gaps sit at rounding level, where the recomputation's own rounding of A v is a
    few percent of them."""
    for (P, b, (_, _, s), run), sigma, tg, th in ((gaps_sigma0, 0.0, 1e-5, 1e-5), (gaps_sigma4, 4.0, 2e-2, 2e-2)):
        A = scipy_of(P)
        g = A @ s["p"] - sigma * s["t"] - s["s"]
        j = A @ s["q"] - s["z"]
        h = A @ s["u"] - sigma * s["r"] - s["w"]
        assert abs(np.linalg.norm(g) - run.gap_g[121]) <= tg * run.gap_g[121], sigma
        assert abs(np.linalg.norm(h) - run.gap_h[122]) <= th * run.gap_h[122], sigma
        assert abs(np.linalg.norm(j) - run.gap_j[121]) <= 2e-2 * run.gap_j[121], sigma
    assert gaps_sigma0[3].gap_g[121] > 100 * gaps_sigma4[3].gap_g[121]     # amplified without the shift


def test_gap_recurrences_of_section_3(gaps_sigma0, gaps_sigma4):
    """The coupled gap recurrences of Section 3.1 on the vectors of consecutive iterations
    (i = 120, 121): each right-hand side reproduces the left-hand side to a few percent of
    the terms it couples, so the local rounding terms are small next to them.
      recur_f: f_{i+1} = f_i - alpha_i g_i + local      (sigma = 0, where g is amplified)
      recur_g: g_i = h_i + beta_i g_{i-1} + local       (sigma = 0 and 4)
      recur_h: h_{i+1} = h_i - alpha_i j_i - alpha_i sigma g_i + local   (sigma = 4)"""
    def parts(data, sigma):
        P, b, (s0, s1, s2), run = data
        A = scipy_of(P)

        def f_of(s):
            return (b - A @ s["x"]) - s["r"]

        def h_of(s):
            return A @ s["u"] - sigma * s["r"] - s["w"]

        def g_of(s):
            return A @ s["p"] - sigma * s["t"] - s["s"]

        return f_of, h_of, g_of, A, (s0, s1, s2), run

    n = np.linalg.norm
    # sigma = 0
    f_of, h_of, g_of, A, (s0, s1, s2), run = parts(gaps_sigma0, 0.0)
    a1, b2 = run.alpha[120], run.beta[121]
    g1, g2 = g_of(s1), g_of(s2)
    assert n(f_of(s1) - (f_of(s0) - a1 * g1)) <= 0.05 * n(a1 * g1)
    assert n(g2 - (h_of(s1) + b2 * g1)) <= 0.05 * (n(h_of(s1)) + n(b2 * g1))
    # sigma = 4: the shift terms of recur_g and recur_h
    f_of, h_of, g_of, A, (s0, s1, s2), run = parts(gaps_sigma4, 4.0)
    a1, b2 = run.alpha[120], run.beta[121]
    g1, g2 = g_of(s1), g_of(s2)
    j1 = A @ s1["q"] - s1["z"]
    assert n(g2 - (h_of(s1) + b2 * g1)) <= 0.1 * (n(h_of(s1)) + n(b2 * g1))
    dh = h_of(s1) - h_of(s0)
    assert n(dh - (-a1 * j1 - a1 * 4.0 * g1)) <= 0.1 * n(dh)
    assert n(a1 * 4.0 * g1) > 0.5 * n(dh)            # the shift's coupling term carries the change


def test_shift_keeps_the_auxiliary_gaps_small():
    """lapl200, 500 iterations: unshifted p-CG amplifies the gap g (Section 3: the propagation
    matrices' norms grow); the shift sigma = 4 of Table 1 keeps every logged gap near the
    rounding level of its first iterations."""
    P, b = S.lapl200()
    p0 = oracle.pcg_sh(P, b, sigma=0.0, maxit=500, log_every=25, gaps=True)
    p4 = oracle.pcg_sh(P, b, sigma=4.0, maxit=500, log_every=25, gaps=True)
    assert np.nanmax(p0.gap_g) > 50 * np.nanmax(p4.gap_g)
    assert np.nanmax(p0.gap) > 1e3 * np.nanmax(p4.gap)
    for v in (p4.gap_g, p4.gap_h, p4.gap_j):
        assert np.nanmax(v) < 1e-12

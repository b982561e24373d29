"""Jacobi M^-1 (Algorithm 3 with its preconditioned recurrences) and the variable
shift of Algorithm 4 on the GPU, against the FP64 oracle, through the C ABI.

Tolerances as in the parity suite: alpha_i, beta_i within 1e-10 relative over
the first 20 iterations; final true relative residual within a factor 10 of
the oracle's.
"""
import numpy as np
import pytest

import oracle
import synthetic as S
from paper_1706_05988_gb300.pcg import PCG_EBREAKDOWN, PCG_ENOTCONV

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


def diag_of(P):
    """diag(A) from the problem description (independent of both sides' operator code)."""
    if P.layout == S.CSR32:
        d = np.zeros(P.n)
        for i in range(P.n):
            lo, hi = P.row_ptr[i], P.row_ptr[i + 1]
            c = P.col[lo:hi]
            d[i] = P.val[lo:hi][c == i].sum()
        return d
    if P.constant:
        return np.full(P.n, 6.0 if P.is_3d else 4.0)
    return np.asarray(P.diag, dtype=np.float64)


def check(g, o, bnorm, k=N_SCALARS, rec_floor=0.0):
    """rec_floor > 0: compare the scalars only while ||r_i|| > rec_floor ||r_0|| (see the p-CG case)."""
    k = min(k, len(o.alpha), len(g.alpha))
    if rec_floor > 0.0:
        k = min(k, int(np.argmax(o.rec / o.rec[0] <= rec_floor)) or k)
    assert k > 0
    assert rel(g.alpha[:k], o.alpha[:k]) <= TOL_SCALARS, (g.alpha[:k], o.alpha[:k])
    assert rel(g.beta[1:k], o.beta[1:k]) <= TOL_SCALARS
    assert g.beta[0] == 0.0
    gt, ot = g.final_true_relres, o.true[-1] / bnorm
    if o.status == 2:
        # stagnation at rounding level ends in a non-positive 1/alpha; where depends on rounding
        assert g.status in (PCG_EBREAKDOWN, PCG_ENOTCONV), g.status
        assert gt <= max(10 * ot, 1e-10), (gt, ot)
    else:
        assert 0.1 * ot <= gt <= 10 * ot, (gt, ot)


def rhs(P, seed=3):
    return S.uniform_pm1(seed, P.n)


PROBLEMS = {
    "varcoef3d_24": lambda: S.varcoef_3d(24, block=4, seed=1),
    "varcoef2d_77x53": lambda: S.varcoef_2d(77, 53, seed=2),
    "lapl3d_20": lambda: S.laplacian_3d(20),
    "csr_sdd_5003": lambda: S.random_sdd_csr(5003, seed=4),
}


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("method,sigma", [("pcg", 0.0), ("spcg", 1.0)])
def test_jacobi_vs_oracle(B, name, method, sigma):
    P = PROBLEMS[name]()
    b = rhs(P)
    maxit = 150
    minv = 1.0 / diag_of(P)
    with B.Solver(P, flags=B.PCG_JACOBI) as s:
        g = s.solve(b, method=method, sigma=sigma, maxit=maxit, true_every=1)
    o = oracle.pcg_sh(P, b, sigma=sigma, maxit=maxit, minv=minv, log_every=1)
    if o.status == 0:
        assert g.iters == o.iters == maxit
    # Unshifted p-CG amplifies local rounding errors (Section 3): on the CSR system, which Jacobi takes
    # to 1e-8 in 19 iterations, the oracle's own sigma = 0 and sigma = 1 runs already differ by 3e-10
    # in alpha_19.  Its scalars are compared while ||r_i|| > 1e-6 ||r_0||.
    check(g, o, np.linalg.norm(b), rec_floor=1e-6 if method == "pcg" else 0.0)


def test_jacobi_converges_like_oracle(B):
    """Stop on ||r_i|| <= tol ||b||: the same iteration (within one) and a comparable true residual."""
    P = S.varcoef_3d(32, block=8, lo_exp=-2, hi_exp=2, seed=5)
    b = rhs(P)
    minv = 1.0 / diag_of(P)
    with B.Solver(P, flags=B.PCG_JACOBI) as s:
        g = s.solve(b, method="spcg", sigma=1.0, tol=1e-8, maxit=2000)
    o = oracle.pcg_sh(P, b, sigma=1.0, rtol=1e-8, maxit=2000, minv=minv, log_every=0)
    assert o.status == 1 and g.status == B.PCG_OK
    assert abs(g.iters - o.iters) <= 1, (g.iters, o.iters)
    assert g.final_true_relres < 1e-7


def test_jacobi_helps_high_contrast(B):
    """On kappa spread over 10^[-3, 3] Jacobi reaches a tolerance unpreconditioned p-CG-sh needs far longer for."""
    P = S.varcoef_3d(32, block=8, seed=6)
    b = rhs(P)
    with B.Solver(P, flags=B.PCG_JACOBI) as s:
        gj = s.solve(b, method="spcg", sigma=1.0, tol=1e-6, maxit=3000)
    with B.Solver(P) as s:
        gi = s.solve(b, method="spcg", sigma=float(np.max(diag_of(P))), tol=1e-6, maxit=3000,
                     raise_on_error=False)
    assert gj.status == B.PCG_OK
    assert gi.status != B.PCG_OK or gi.iters > 2 * gj.iters


def test_jacobi_x0_and_zero_rhs(B):
    P = S.varcoef_2d(40, 33, seed=7)
    b = rhs(P)
    x0 = S.uniform_pm1(8, P.n)
    minv = 1.0 / diag_of(P)
    with B.Solver(P, flags=B.PCG_JACOBI) as s:
        g = s.solve(b, x0=x0, method="spcg", sigma=1.0, maxit=60, true_every=1)
        z = s.solve(np.zeros(P.n), method="spcg", sigma=1.0, maxit=60)
    o = oracle.pcg_sh(P, b, x0=x0, sigma=1.0, maxit=60, minv=minv, log_every=1)
    check(g, o, np.linalg.norm(b))
    # b = 0, x0 = 0: (r_0, u_0) = 0, the iteration stops before its first step with x = 0
    assert z.iters == 0 and z.status == B.PCG_OK and not np.any(z.x)


def test_jacobi_deterministic(B):
    P = S.random_sdd_csr(20011, seed=9)
    b = rhs(P)
    with B.Solver(P, flags=B.PCG_JACOBI) as s:
        g1 = s.solve(b, method="spcg", sigma=1.0, maxit=80)
        g2 = s.solve(b, method="spcg", sigma=1.0, maxit=80)
    assert np.array_equal(g1.x, g2.x) and np.array_equal(g1.alpha, g2.alpha)


# ------------------------------------------------------------------ variable shift (Algorithm 4)

def schedule(maxit, hi, lo, seed=0):
    """A shift that starts at hi and decays towards lo (plus a seeded jitter), hi >= sigma >= lo >= 0."""
    k = np.arange(maxit + 1)
    j = 0.05 * S.uniform01(seed, maxit + 1)
    return lo + (hi - lo) * np.exp(-k / 30.0) * (1.0 + j) / 1.05


@pytest.mark.parametrize("name,jacobi", [("lapl3d_20", False), ("varcoef2d_77x53", False),
                                         ("varcoef3d_24", True), ("csr_sdd_5003", True)])
def test_varshift_vs_oracle(B, name, jacobi):
    P = PROBLEMS[name]()
    b = rhs(P)
    maxit = 120
    minv = 1.0 / diag_of(P) if jacobi else None
    hi = 1.0 if jacobi else float(np.max(diag_of(P)))
    sh = schedule(maxit, hi, 0.1 * hi, seed=11)
    with B.Solver(P, flags=B.PCG_JACOBI if jacobi else 0) as s:
        assert B.pcg_set_shifts(s.ctx, sh) == B.PCG_OK
        g = s.solve(b, method="spcg", sigma=123.0, maxit=maxit, true_every=1)   # sigma ignored
    o = oracle.pcg_varsh(P, b, sh, maxit=maxit, minv=minv, log_every=1)
    check(g, o, np.linalg.norm(b))


def test_constant_schedule_is_algorithm3(B):
    """A constant schedule is Algorithm 3: it runs the constant-shift kernel, bit for bit."""
    P = S.laplacian_3d(24)
    b = rhs(P)
    sh = np.full(101, 6.0)
    with B.Solver(P) as s:
        assert B.pcg_set_shifts(s.ctx, sh) == B.PCG_OK
        g = s.solve(b, method="spcg", maxit=100, true_every=1)
        assert B.pcg_set_shifts(s.ctx, None) == B.PCG_OK
        f = s.solve(b, method="spcg", sigma=6.0, maxit=100, true_every=1)   # the fused constant-shift path
    o = oracle.pcg_sh(P, b, sigma=6.0, maxit=100, log_every=1)
    check(g, o, np.linalg.norm(b))
    check(f, o, np.linalg.norm(b))
    assert np.array_equal(g.x, f.x) and np.array_equal(g.alpha, f.alpha)


def test_general_errors(B):
    P = S.laplacian_2d(32)
    b = rhs(P)
    with B.Solver(P, flags=B.PCG_JACOBI) as s:
        r = s.solve(b, method="cg", maxit=10, precision=B.PCG_MIXED_IR, raise_on_error=False)
        assert r.status == B.PCG_ENOTIMPL
        assert B.pcg_set_shifts(s.ctx, np.array([1.0, -0.5])) == B.PCG_EINVAL
        assert B.pcg_set_shifts(s.ctx, np.array([1.0, np.nan])) == B.PCG_EINVAL
        assert B.pcg_set_shifts(s.ctx, np.full(5, 1.0)) == B.PCG_OK
        r = s.solve(b, method="spcg", maxit=10, raise_on_error=False)   # needs maxit + 1 = 11 shifts
        assert r.status == B.PCG_EINVAL
        r = s.solve(b, method="spcg", maxit=4)
        assert r.status in (B.PCG_OK, B.PCG_ENOTCONV) and r.iters == 4


def test_psi_varsh_matches_oracle(B):
    """psi_i of Section 4.1 (variable shift) on the device against the oracle, for constant,
    ramped, decaying and jittered schedules over lapl200's history; a constant schedule also
    equals pcg_psi's constant-shift value."""
    from oracle import psi as PS
    from paper_1706_05988_gb300 import pcg as C
    P, b = S.lapl200()
    o = oracle.pcg_sh(P, b, sigma=4.0, maxit=301, log_every=0)
    i = 300
    k = np.arange(i + 2)
    scheds = np.stack([np.full(i + 2, 4.0), 4.0 * k / (i + 1), 2.0 + 4.0 * np.exp(-k / 50.0),
                       4.0 + 0.5 * (S.uniform01(5, i + 2) - 0.5)])
    with B.Solver(P) as s:
        g = C.pcg_psi_varsh(s.ctx, o.alpha, o.beta, i, scheds)
        g4 = C.pcg_psi(s.ctx, o.alpha, o.beta, i, np.array([4.0]))
    ref = np.array([PS.psi_varsh(o.alpha, o.beta, i, sc) for sc in scheds])
    assert rel(g, ref) < 1e-9, (g, ref)
    assert rel(g[:1], g4) < 1e-12
    with B.Solver(P) as s:
        with pytest.raises(C.PcgError):
            C.pcg_psi_varsh(s.ctx, o.alpha, o.beta, i, scheds[:, :i + 1])   # too short a schedule


def test_jacobi_with_device_matrix_arrays(B):
    """PCG_JACOBI on matrices given as device arrays: D^-1 is formed on the device and the solve
    is bit-identical to the one from host arrays (variable-coefficient stencil and CSR); a zero
    diagonal on the device is rejected."""
    import torch
    from paper_1706_05988_gb300 import pcg as C
    P = S.varcoef_3d(16, block=4, seed=8)
    dev = {k: torch.from_numpy(getattr(P, k)).cuda() for k in ("diag", "ax", "ay", "az")}
    b = S.normal(4, P.n)
    with B.Solver(P, flags=B.PCG_JACOBI) as s1, B.Solver(P, flags=B.PCG_JACOBI, device_arrays=dev) as s2:
        r1 = s1.solve(b, method="spcg", sigma=1.0, maxit=40)
        r2 = s2.solve(b, method="spcg", sigma=1.0, maxit=40)
    assert np.array_equal(r1.x, r2.x) and np.array_equal(r1.alpha, r2.alpha)
    Q = S.random_sdd_csr(3001, seed=12)
    devc = {"row_ptr": torch.from_numpy(Q.row_ptr).cuda(), "col": torch.from_numpy(Q.col).cuda(),
            "val": torch.from_numpy(Q.val).cuda()}
    bq = S.normal(5, Q.n)
    with B.Solver(Q, flags=B.PCG_JACOBI) as s1, B.Solver(Q, flags=B.PCG_JACOBI, device_arrays=devc) as s2:
        r1 = s1.solve(bq, method="spcg", sigma=1.0, maxit=25)
        r2 = s2.solve(bq, method="spcg", sigma=1.0, maxit=25)
    assert np.array_equal(r1.x, r2.x)
    bad = dict(dev)
    bad["diag"] = dev["diag"].clone()
    bad["diag"][7] = 0.0
    with pytest.raises(C.PcgError):
        B.Solver(P, flags=B.PCG_JACOBI, device_arrays=bad)


@pytest.mark.parametrize("name", ["varcoef3d_24", "varcoef2d_77x53", "csr_sdd_5003"])
def test_jacobi_cg_vs_oracle(B, name):
    """Algorithm 1 with M^-1 = D^-1 (the paper's JAC rows of Table 1) against the oracle's CG."""
    P = PROBLEMS[name]()
    b = rhs(P)
    minv = 1.0 / diag_of(P)
    with B.Solver(P, flags=B.PCG_JACOBI) as s:
        g = s.solve(b, method="cg", maxit=150, true_every=1)
        t = s.solve(b, method="cg", tol=1e-9, maxit=5000)
    o = oracle.cg(P, b, maxit=150, minv=minv, log_every=1)
    ot = oracle.cg(P, b, maxit=5000, rtol=1e-9, minv=minv, log_every=0)
    check(g, o, np.linalg.norm(b), rec_floor=1e-6)
    assert t.status == B.PCG_OK and ot.status == 1 and abs(t.iters - ot.iters) <= 1, (t.iters, ot.iters)


def test_varcoef_128_jacobi_full_size_vs_oracle(B):
    """The 128^3 high-contrast FV system (kappa = 10^U[-3,3] on 8^3 blocks, b ~ N(0,1)) at full size:
    Jacobi shifted p-CG's first 20 iterations against the oracle, and the mixed-precision form with
    binary64 refinement reaching a true relative residual of 1e-10, checked by the oracle's operator."""
    P = S.varcoef_3d(128, block=8, seed=0)
    b = S.normal(1, P.n)
    minv = 1.0 / diag_of(P)
    with B.Solver(P, flags=B.PCG_JACOBI) as s:
        g = s.solve(b, method="spcg", sigma=1.0, maxit=20, true_every=0)
        m = s.solve(b, method="spcg", sigma=1.0, tol=1e-10, maxit=40000, precision=B.PCG_MIXED_IR)
    o = oracle.pcg_sh(P, b, sigma=1.0, maxit=20, minv=minv, log_every=0)
    assert g.iters == o.iters == 20
    assert rel(g.alpha[:20], o.alpha[:20]) <= TOL_SCALARS
    assert rel(g.beta[1:20], o.beta[1:20]) <= TOL_SCALARS
    idx = np.random.default_rng(2).integers(0, P.n, 20000)
    np.testing.assert_allclose(g.x[idx], o.x[idx], rtol=1e-9, atol=1e-11 * np.abs(o.x).max())
    assert m.status == B.PCG_OK
    bn = np.linalg.norm(b)
    assert np.linalg.norm(b - oracle.apply(P, m.x)) <= 1.05e-10 * bn


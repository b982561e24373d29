"""One system split into z-slabs, with the slab kernels of the C ABI (pcg_slab_*), GB300
only.  The slabs of every rank are held by this process on one GPU and stepped phase by
phase (sharded.solve_local): halo planes and the dot reduction are copies between their
tensors, so no kernel ever waits for another.  The result must be the oracle's Algorithm 3
on the whole grid: alpha_i, beta_i to 1e-10 over 20 iterations, every entry of x, and the
true residual."""
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
    return np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b))


def sharded_run(grid, world, sigma, maxit, tol=0.0, seed=31):
    from paper_1706_05988_gb300 import sharded as SH
    nx, ny, nz = grid
    P = S.laplacian_3d(nx, ny, nz)
    b = S.normal(seed, P.n)
    slabs = []
    for k0, k1 in SH.z_slabs(nz, world):
        slabs.append(SH.CudaSlab(nx, ny, k0, k1, nz, b[k0 * nx * ny:k1 * nx * ny], maxit))
    res = SH.solve_local(slabs, sigma, tol, maxit, check_every=0 if tol == 0 else 25)
    hist = [s.history(maxit + 1) for s in slabs]
    x = np.concatenate([s.x_host() for s in slabs])
    for s in slabs:
        s.close()
    return P, b, res, hist, x


CASES = [((32, 30, 29), 2), ((32, 30, 29), 3), ((31, 20, 17), 2), ((16, 16, 4), 4), ((40, 36, 33), 4)]


@pytest.mark.parametrize("grid,world", CASES, ids=[f"{g[0]}x{g[1]}x{g[2]}_w{w}" for g, w in CASES])
def test_sharded_slabs_vs_oracle(B, grid, world):
    maxit, sigma = 20, 6.0
    P, b, res, hist, x = sharded_run(grid, world, sigma, maxit)
    o = oracle.pcg_sh(P, b, sigma=sigma, maxit=maxit, log_every=maxit)
    assert res["iters"] == maxit and res["status"] == B.PCG_ENOTCONV
    for a, bt, _ in hist:                         # every slab holds the same global scalars
        assert np.all(rel(a[:maxit], o.alpha) <= 1e-10)
        assert bt[0] == 0.0 and np.all(rel(bt[1:maxit], o.beta[1:]) <= 1e-10)
    scale = np.abs(o.x).max()
    assert np.all(np.abs(x - o.x) <= 1e-10 * np.abs(o.x) + 1e-12 * scale)
    bn = np.linalg.norm(b)
    assert abs(res["true_relres"] - o.true[-1] / bn) <= 1e-8 * o.true[-1] / bn


def test_sharded_converges_like_single_solver(B):
    """To a tolerance: the same stop iteration as the single-system solver (within 1) and a
    true residual at the tolerance."""
    grid = (48, 44, 40)
    P, b, res, hist, x = sharded_run(grid, 3, 6.0, 2000, tol=1e-10)
    with B.Solver(P) as s:
        g = s.solve(b, method="spcg", sigma=6.0, tol=1e-10, maxit=2000)
    assert res["status"] == B.PCG_OK and g.status == B.PCG_OK
    assert abs(res["iters"] - g.iters) <= 1
    assert res["true_relres"] <= 2e-10
    assert np.linalg.norm(x - g.x) <= 1e-8 * np.linalg.norm(g.x)

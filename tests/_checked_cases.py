"""Runs a set of solves through the library that PCG_LIBRARY names (or the default one) and
saves their results to the .npz file given as the only argument, with the index-check
status of the run.  Used by test_gpu_checked.py to run the same cases with the ordinary
and the index-checked build (libpcg_checked.so)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402


def main(out_path):
    import torch
    import paper_1706_05988_gb300 as pkg
    from paper_1706_05988_gb300 import pcg as C
    from paper_1706_05988_gb300 import sharded as SH
    res = {}

    def solve(name, P, sigma, maxit, flags=0, precision=C.PCG_FP64, tol=0.0, stages=None, shifts=None):
        b = S.normal(5, P.n)
        with pkg.Solver(P, flags=flags) as s:
            if stages is not None:
                assert C.pcg_set_param(s.ctx, C.PCG_PARAM_ITER_STAGES, float(stages)) == C.PCG_OK
            if shifts is not None:
                assert C.pcg_set_shifts(s.ctx, shifts) == C.PCG_OK
            r = s.solve(b, method="spcg", sigma=sigma, maxit=maxit, tol=tol, precision=precision, true_every=5)
        res[name + "_x"] = r.x
        res[name + "_alpha"] = r.alpha

    solve("st3d_even", S.laplacian_3d(20, 18, 16), 6.0, 30)
    solve("st3d_odd", S.laplacian_3d(15, 17, 9), 6.0, 30)
    solve("st2d_odd", S.laplacian_2d(37, 23), 4.0, 30)
    solve("st2d_even", S.laplacian_2d(64, 45), 4.0, 30)
    solve("var3d_odd", S.varcoef_3d(17, block=4, seed=4), 1.0, 30)
    solve("var2d_even", S.varcoef_2d(48, 40, seed=1), 1.0, 30)
    solve("csr_lapl", S.to_csr(S.laplacian_3d(18, 14, 10)), 6.0, 30)
    solve("csr_sdd", S.random_sdd_csr(3001, seed=3), 2.0, 30)
    solve("jacobi_var3d", S.varcoef_3d(24, block=8, seed=3), 1.0, 30, flags=C.PCG_JACOBI)
    solve("mixed_lapl", S.laplacian_3d(24), 6.0, 400, precision=C.PCG_MIXED_IR, tol=1e-9)
    solve("mixed_jacobi", S.varcoef_3d(24, block=8, seed=3), 1.0, 2000, flags=C.PCG_JACOBI,
          precision=C.PCG_MIXED_IR, tol=1e-8)
    solve("varshift", S.laplacian_3d(16), 0.0, 30, shifts=np.linspace(1.0, 5.0, 31))
    solve("staged2", S.laplacian_3d(34, 30, 7), 6.0, 30, stages=2)
    solve("staged3_2d", S.laplacian_2d(100, 70), 4.0, 30, stages=3)
    solve("persistent", S.laplacian_3d(32), 6.0, 30, flags=C.PCG_PERSISTENT)
    # batch and server
    probs = [S.varcoef_2d(int(a), int(a) + 3, seed=i) for i, a in enumerate((20, 45, 90, 130))]
    bs = [S.normal(40 + i, P.n) for i, P in enumerate(probs)]
    with pkg.Batch(probs, flags=C.PCG_JACOBI) as bt:
        xs, it, st, tr = bt.solve(bs, [1.0] * 4, tol=1e-8, maxit=4000)
    for i, x in enumerate(xs):
        res[f"batch{i}_x"] = x
    with pkg.Server(1 << 30, 8) as srv:
        P = S.random_sdd_csr(4000, seed=8)
        t = srv.submit(P, S.normal(9, P.n), tol=1e-9, method=C.PCG_SPCG, sigma=2.0)
        r = None
        while r is None:
            r = srv.poll(t)
        res["served_x"] = r[1]
    # one system in three slabs, stepped in this process
    nx, ny, nz = 18, 16, 15
    bb = S.normal(12, nx * ny * nz)
    slabs = [SH.CudaSlab(nx, ny, k0, k1, nz, bb[k0 * nx * ny:k1 * nx * ny], 30) for k0, k1 in SH.z_slabs(nz, 3)]
    SH.solve_local(slabs, 6.0, 0.0, 30, check_every=0)
    res["slabs_x"] = np.concatenate([s.x_host() for s in slabs])
    for s in slabs:
        s.close()
    torch.cuda.synchronize()
    code, checked = C.pcg_check_status()
    res["check_code"] = np.array([code])
    res["checked_build"] = np.array([int(checked)])
    np.savez(out_path, **res)


if __name__ == "__main__":
    main(sys.argv[1])

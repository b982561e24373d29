"""Writes the full-size oracle fixtures of tests/golden/ (calls only oracle/ and synthetic/).

    python tests/golden/make_full_size_golden.py            # all cases, in parallel processes
    python tests/golden/make_full_size_golden.py spcg_256   # one case

Cases (each a plain single-threaded oracle run; minutes each):
  spcg_256      shifted p-CG (Algorithm 3), sigma = 6, 1,000 iterations on the 256^3 7-point
                Laplacian, b = A x* with dyadic x* ~ U[-1,1] (seed 0), x0 = 0, M = I
  spcg_256_csr  the same system assembled as CSR with int32 indices
  varcoef_128   Algorithm 3 with Jacobi M^-1 = D^-1, sigma = 0.75, on the 128^3 FV diffusion
                problem (kappa = 10^U[-3,3] on 8^3 blocks, seed 0), b ~ N(0,1) (stream 1), x0 = 0,
                stopped once ||r_i|| <= 1e-10 ||b|| (Section 5.2's scaled criterion)

Each fixture stores what the GPU tests compare against: the final true relative residual
||b - A x|| / ||b|| of the last iterate, the recursive residual path, alpha_i and beta_i of the
first 20 iterations and of every 50th, and (varcoef_128) the iterate at 4,096 seeded indices.
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ITERS_256 = 1000
SIGMA_256 = 6.0
SIGMA_VARCOEF = 0.75
RTOL_VARCOEF = 1e-10
SAMPLE_SEED = 7          # numpy generator seed of the sampled indices of x
SAMPLE_COUNT = 4096

OUT = {
    "spcg_256": os.path.join(HERE, "spcg_256cubed_1000it.json"),
    "spcg_256_csr": os.path.join(HERE, "spcg_256cubed_csr_1000it.json"),
    "varcoef_128": os.path.join(HERE, "varcoef128_jacobi_spcg_1e-10.json"),
}


def _scalars(run, every=50, first=20):
    idx = sorted(set(range(min(first, run.iters))) | set(range(0, run.iters, every)))
    return {"index": idx, "alpha": [float(run.alpha[i]) for i in idx], "beta": [float(run.beta[i]) for i in idx]}


def _rec_path(run, bnorm, every=50):
    return {"index": list(range(0, run.iters + 1, every)),
            "rec_relres": [float(run.rec[i] / bnorm) for i in range(0, run.iters + 1, every)]}


def case_spcg_256(csr: bool) -> dict:
    import numpy as np
    import oracle
    import synthetic as S
    P, b, _ = S.poisson3d_manufactured(256)
    if csr:
        P = S.to_csr(P)
    bn = float(np.linalg.norm(b))
    t0 = time.time()
    o = oracle.pcg_sh(P, b, sigma=SIGMA_256, maxit=ITERS_256, log_every=10 * ITERS_256)
    dt = time.time() - t0
    return {
        "what": ("oracle p-CG-sh (Algorithm 3), sigma = 6, 1,000 iterations, 256^3 7-point Laplacian"
                 + (" as CSR int32" if csr else " (matrix-free)")
                 + "; b = A x*, x* dyadic U[-1,1] seed 0, x0 = 0, M = I"),
        "written_by": "tests/golden/make_full_size_golden.py (oracle/ only)",
        "n": int(P.n), "iters": int(o.iters), "status": int(o.status), "bnorm": bn,
        "final_true_relres": float(o.true[-1] / bn),
        "final_rec_relres": float(o.rec[-1] / bn),
        "final_gap_rel": float(o.gap[-1] / bn),
        "rec_path": _rec_path(o, bn),
        "scalars": _scalars(o),
        "oracle_seconds": dt,
    }


def case_varcoef_128() -> dict:
    import numpy as np
    import oracle
    import synthetic as S
    P = S.varcoef_3d(128, block=8, seed=0)
    b = S.normal(1, P.n)
    bn = float(np.linalg.norm(b))
    minv = 1.0 / np.asarray(P.diag, dtype=np.float64)
    t0 = time.time()
    o = oracle.pcg_sh(P, b, sigma=SIGMA_VARCOEF, maxit=40000, rtol=RTOL_VARCOEF, minv=minv, log_every=10 ** 9)
    dt = time.time() - t0
    idx = np.sort(np.random.default_rng(SAMPLE_SEED).choice(P.n, SAMPLE_COUNT, replace=False))
    return {
        "what": ("oracle p-CG-sh (Algorithm 3) with Jacobi M^-1, sigma = 0.75, to ||r_i|| <= 1e-10 ||b||; "
                 "128^3 FV diffusion, kappa 10^U[-3,3] on 8^3 blocks (seed 0), b ~ N(0,1) stream 1, x0 = 0"),
        "written_by": "tests/golden/make_full_size_golden.py (oracle/ only)",
        "n": int(P.n), "iters": int(o.iters), "status": int(o.status), "bnorm": bn,
        "final_true_relres": float(o.true[-1] / bn),
        "final_rec_relres": float(o.rec[-1] / bn),
        "x_norm": float(np.linalg.norm(o.x)),
        "x_sample": {"numpy_rng_seed": SAMPLE_SEED, "count": SAMPLE_COUNT,
                     "index": [int(i) for i in idx], "value": [float(v) for v in o.x[idx]]},
        "rec_path": _rec_path(o, bn, every=250),
        "scalars": _scalars(o),
        "oracle_seconds": dt,
    }


def run_case(name: str) -> str:
    if name == "spcg_256":
        d = case_spcg_256(False)
    elif name == "spcg_256_csr":
        d = case_spcg_256(True)
    elif name == "varcoef_128":
        d = case_varcoef_128()
    else:
        raise SystemExit(f"unknown case {name}")
    with open(OUT[name], "w") as f:
        json.dump(d, f, indent=1)
        f.write("\n")
    return f"{name}: {d['iters']} iterations, final true relres {d['final_true_relres']:.3e} " \
           f"({d['oracle_seconds']:.0f} s) -> {os.path.relpath(OUT[name], ROOT)}"


def main(argv):
    names = argv or list(OUT)
    import oracle
    oracle.build()
    if len(names) == 1:
        print(run_case(names[0]))
        return
    with mp.get_context("spawn").Pool(len(names)) as pool:
        for line in pool.imap_unordered(run_case, names):
            print(line, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])

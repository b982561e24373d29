"""Benchmark: shifted pipelined CG (arXiv 1706.05988, Algorithm 3) on the 256^3
7-point Laplacian in FP64, through the C ABI of libpcg.

One step = one solve of 1,000 p-CG-sh iterations (sigma = 6, b = A x*, x0 = 0).
value = iterations/s over all ranks with the step's inputs resident in HBM;
e2e = the same through pcg_solve with host buffers (pinned), H2D of b and D2H
of x inside the timed region.  Each rank solves its own system (independent
problems: no data-path collective).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# The headline metric names both halves; `value` is the first (iterations/s of the 256^3
# FP64 solve, with its HBM GB/s in `roofline` and `hbm_gbs_effective`); the served
# solves/s and p99 at a relative residual of 1e-8 are the `serving_tol_1e-8` object.
METRIC = "p-CG iters/s & HBM GB/s (256³ FP64); served solves/s, p99 at ≤1e-8 rel. res"
UNIT = "iter/s"
N_SIDE = 256                # overridable with --size (profiling captures use a smaller grid)
ITERS_PER_STEP = 1000
SIGMA = 6.0
BYTES_PER_DOF = 96          # x, r, w, z, s, p: one FP64 read + one FP64 write each per iteration
FP64_OPS_PER_DOF = 9        # DFMA per unknown per fused iteration (the stencil row runs on the integer pipe)
FALLBACK_HBM_GBS = 6800.0

# k_spcg_iter<StencilOp<3, ST_LAP_FIXED, 2>> on 256^3: dram__bytes_read.sum + dram__bytes_write.sum of one launch
# (a one-pass capture, profiles/spcg_iter_stencil7_256cubed_traffic.md), keyed by the SHA-256 of the kernel
# source it was taken on; a changed kernel reports null
NCU_TRAFFIC = {"db28dd47f9fa25b7": 1561.35e6, "e9be0f27e77e4297": 1561.47e6, "9a4ca33e0286f39c": 1561.25e6,
               "a8b0005e527d5aff": 1561.77e6, "ed0a31d47b72680c": 1561.46e6,
               "bbd2e5118c8fc4ca": 1561.30e6}


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in ("pcg_kernels.cuh", "pcg_fixedsum.cuh", "pcg_kernels_3d.cu"):
        with open(os.path.join(ROOT, "paper_1706_05988_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def workload_config(n: int) -> dict:
    return {"workload": f"3D 7-point constant-coefficient Dirichlet Laplacian on {N_SIDE}^3 (n={n:,}), matrix-free "
                        f"stencil; shifted p-CG (Alg. 3) sigma={SIGMA}, {ITERS_PER_STEP} iterations per step; "
                        "b = A x*, x* ~ U[-1,1] (seed 0), x0 = 0",
            "n": n, "iterations_per_step": ITERS_PER_STEP, "sigma": SIGMA,
            "l2": "inputs larger than L2 (six 128 MiB FP64 vectors streamed per iteration)"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]), f[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def dist_setup(gpus: int, backend: str = "nccl"):
    """Rank, world size and local rank from the torchrun environment; joins the process group
    when there is more than one rank (NCCL on the GPUs; gloo for the host-side tests)."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != gpus:
        raise SystemExit(f"--gpus {gpus} but WORLD_SIZE {world}")
    if world > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: every rank's units (independent systems, no data-path
    collective) over the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)


def cpu_oracle_rate(P, b, iters: int, omp: bool = False) -> tuple[float, float]:
    """Iterations/s of the oracle's Algorithm 3 on (P, b): the single-threaded parity build,
    or (omp) the same source built with OpenMP, on every host core."""
    import oracle
    oracle.build(omp=omp)
    if omp:
        oracle.threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    oracle.pcg_sh(P, b, sigma=SIGMA, maxit=iters, log_every=0, omp=omp)
    dt = time.perf_counter() - t0
    return iters / dt, dt


# Algorithmic bytes per unknown and iteration of the per-cluster solvers on 2D variable-
# coefficient systems (vectors and face coefficients read once and written once per sweep):
#   fp64 (M = I): reads w, 3 coefficient arrays, z, s, p, r, x (72 B); writes z, s, p, x, r, w' (48 B)
#   fp64_jacobi: reads m, 3 coefficients, w, r, u, t, s, z, p, q, x, D^-1 (112 B); writes t, s, z,
#                p, q, x, r, u, w', m' (80 B)
#   mixed_jacobi: binary32 m, 3 coefficients, w, z, s, p, u, t, q, D^-1 and binary64 r, x (64 B);
#                 writes binary32 z, s, p, u, t, q, w', m' and binary64 r, x (48 B)
# Small systems keep their vectors in L2, so these are algorithmic, not DRAM, bytes.
BATCH_BYTES_PER_UNKNOWN_ITER = {"fp64": 120, "fp64_jacobi": 192, "mixed_jacobi": 112}


def batch_measure(pkg, S, nsys: int, side_hi: int, forms=("fp64_jacobi", "mixed_jacobi"), seed: int = 0,
                  peak_gbs: float = None) -> dict:
    """Solves/s of nsys 2D FV systems (sides U{32..side_hi}, kappa = 10^U[-2,2] per cell, b ~ N(0,1),
    tol 1e-8) in one batched launch, in the given forms: `fp64` (M = I, sigma = half the median
    diagonal), `fp64_jacobi` and `mixed_jacobi` (Jacobi M^-1, sigma = 1; mixed precision with FP64
    refinement); against plain FP64 solves one at a time through the single-system entry point
    (a sample of 16 systems), all through host buffers."""
    import numpy as np
    import torch
    from paper_1706_05988_gb300 import pcg as C
    rng = np.random.default_rng(seed)
    sides = rng.integers(32, side_hi + 1, size=nsys)
    probs = [S.varcoef_2d(int(L), int(L), seed=seed + i) for i, L in enumerate(sides)]
    bs = [S.normal(1000 + i, P.n) for i, P in enumerate(probs)]
    sig_plain = [0.5 * float(np.median(P.diag)) for P in probs]
    out = {"workload": f"{nsys} 2D variable-coefficient 5-point systems, sides U{{32..{side_hi}}}, kappa 10^U[-2,2] "
                       "per cell, b ~ N(0,1), tol 1e-8"}
    kinds = {"fp64": (0, C.PCG_FP64, sig_plain), "fp64_jacobi": (pkg.PCG_JACOBI, C.PCG_FP64, [1.0] * nsys),
             "mixed_jacobi": (pkg.PCG_JACOBI, C.PCG_MIXED_IR, [1.0] * nsys)}
    for name in forms:
        flags, prec, sig = kinds[name]
        with pkg.Batch(probs, flags=flags, precision=prec) as bt:
            c, _ = bt.autotune(bs, sig, probe_iters=50)
            bt.solve(bs, sig, tol=1e-8, maxit=100000)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, it, st, tr = bt.solve(bs, sig, tol=1e-8, maxit=100000)
            torch.cuda.synchronize()
            tb = time.perf_counter() - t0
            out[name] = {"solves_per_s": nsys / tb, "kernel_ms": bt.last_kernel_ms(), "uniform_cluster_size": c,
                         "converged": int(np.sum(st == 0)), "max_true_relres": float(np.max(tr)),
                         "mean_iters": float(np.mean(it)),
                         "unknown_iterations": float(np.sum(it.astype(np.float64) * np.array([P.n for P in probs])))}
            ui_s = out[name]["unknown_iterations"] / tb
            gbs = ui_s * BATCH_BYTES_PER_UNKNOWN_ITER[name] / 1e9
            out[name].update({"unknown_iterations_per_s": ui_s, "algorithmic_gbs": gbs,
                              "bytes_per_unknown_iteration": BATCH_BYTES_PER_UNKNOWN_ITER[name]})
            if peak_gbs:
                out[name]["frac_of_hbm"] = gbs / peak_gbs
    k = min(nsys, 16)
    idx = np.linspace(0, nsys - 1, k).astype(int)
    t1 = 0.0
    for i in idx:
        with pkg.Solver(probs[i]) as one:
            one.solve(bs[i], method="spcg", sigma=sig_plain[i], tol=1e-8, maxit=100000)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            one.solve(bs[i], method="spcg", sigma=sig_plain[i], tol=1e-8, maxit=100000)
            torch.cuda.synchronize()
            t1 += time.perf_counter() - t0
    one_rate = k / t1
    out["one_at_a_time_fp64"] = {"solves_per_s": one_rate, "sample": int(k)}
    for name in forms:
        out["speedup_" + name] = out[name]["solves_per_s"] / one_rate
    return out


def varcoef_measure(pkg, S) -> dict:
    """128^3 FV diffusion, kappa = 10^U[-3,3] on 8^3 blocks, b ~ N(0,1), to a true relative residual
    of 1e-10 with Jacobi: FP64 shifted p-CG against mixed precision with FP64 refinement (the same
    shift, from the psi tool over a 30-iteration pilot), each timed once after a warm-up solve."""
    import ctypes
    import numpy as np
    import torch
    from paper_1706_05988_gb300 import pcg as C
    P = S.varcoef_3d(128, block=8, seed=0)
    b = S.normal(1, P.n)
    out = {"workload": "128^3 7-point FV diffusion, kappa 10^U[-3,3] on 8^3 blocks, b ~ N(0,1), Jacobi M^-1, "
                       "tol 1e-10 (true residual)"}
    with pkg.Solver(P, flags=pkg.PCG_JACOBI) as s:
        grid = np.linspace(0.0, 2.0, 41)
        so = ctypes.c_double()
        st = C.lib().pcg_select_sigma(s.ctx, np.ascontiguousarray(b).ctypes.data, 30, grid.ctypes.data, grid.size,
                                      ctypes.byref(so), None)
        sigma = so.value if st == C.PCG_OK else 1.0
        out["sigma"] = sigma
        for name, prec in (("fp64", C.PCG_FP64), ("mixed_ir", C.PCG_MIXED_IR)):
            for rep in range(2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = s.solve(b, method="spcg", sigma=sigma, tol=1e-10, maxit=40000, precision=prec,
                            raise_on_error=False)
                dt = time.perf_counter() - t0
            out[name] = {"ms": dt * 1e3, "iters": int(r.iters), "status": int(r.status),
                         "true_relres": float(r.final_true_relres)}
            # whole-solve algorithmic rate: iterations x n x the sweep's bytes per unknown (binary64
            # Jacobi: 21 vector accesses + 4 coefficient arrays = 200 B; mixed Jacobi: 104 B of
            # vectors + 4 binary32 coefficient arrays = 120 B); restarts and polling included
            bpu = 200 if name == "fp64" else 120
            out[name]["algorithmic_gbs"] = r.iters * P.n * bpu / dt / 1e9
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms"] / out["mixed_ir"]["ms"]
    return out


def serving_trace(nreq: int, rate: float, seed: int = 0, n_max_exp: float = 5.0, first: int = None):
    """Seeded request stream: Poisson arrivals at `rate` per second; n log-uniform in
    [1e3, 10^n_max_exp]; half stencils (2D/3D unscaled Laplacians), half random SDD CSR (7-27
    entries per row, off-diagonals U[-1,0]); tolerance log-uniform in [1e-10, 1e-6]; b ~ N(0,1).
    first: build only the first requests of the same stream."""
    import numpy as np
    import synthetic as S
    u = S.uniform01(seed, 4 * nreq).reshape(nreq, 4)
    gaps = -np.log(1.0 - u[:, 0]) / rate
    arrive = np.cumsum(gaps)
    reqs = []
    for i in range(nreq if first is None else min(first, nreq)):
        n = int(10 ** (3 + (n_max_exp - 3) * u[i, 1]))
        if u[i, 2] < 0.25:
            side = max(int(round(n ** 0.5)), 4)
            P = S.laplacian_2d(side)
        elif u[i, 2] < 0.5:
            side = max(int(round(n ** (1 / 3))), 4)
            P = S.laplacian_3d(side)
        else:
            P = S.random_sdd_csr(n, seed=seed + 100 + i)
        tol = 10 ** (-10 + 4 * u[i, 3])
        reqs.append((arrive[i], P, S.normal(seed + 10000 + i, P.n), tol))
    return reqs


def request_policy(P, form: str):
    """Per-request (flags, precision) of a served form.  `fp64`: binary64, M = I.
    `mixed`: mixed precision with binary64 refinement; M = I on the constant-coefficient
    stencils (their diagonal is constant, so Jacobi would only rescale them while adding
    the D^-1 traffic), Jacobi M^-1 on CSR (diagonals that vary from row to row).
    `mixed_jacobi`: mixed precision with Jacobi on every request."""
    import paper_1706_05988_gb300 as pkg
    from paper_1706_05988_gb300 import pcg as C
    if form == "fp64":
        return 0, C.PCG_FP64
    if form == "mixed_jacobi" or P.layout == 2:
        return pkg.PCG_JACOBI, C.PCG_MIXED_IR
    return 0, C.PCG_MIXED_IR


def serve_stream(pkg, reqs, form: str):
    """Runs the request stream through one server with the form's per-request policy;
    returns (latencies, span).  The client's garbage collector is paused inside the timed
    loop (as in the one-at-a-time arm): a collection there would stop the submissions and
    polls that drive the server."""
    import gc
    import numpy as np
    nreq = len(reqs)
    lat = np.zeros(nreq)
    gc.collect()
    gc.disable()
    try:
        return _serve_stream(pkg, reqs, form, lat)
    finally:
        gc.enable()


def _serve_stream(pkg, reqs, form, lat):
    nreq = len(reqs)
    with pkg.Server(8 << 30, 512) as srv:
        pending = {}
        t0 = time.perf_counter()
        i = 0
        done = 0
        while done < nreq:
            now = time.perf_counter() - t0
            while i < nreq and reqs[i][0] <= now:
                flags, prec = request_policy(reqs[i][1], form)
                pending[srv.submit(reqs[i][1], reqs[i][2], tol=reqs[i][3], flags=flags, precision=prec)] = i
                i += 1
            for t in list(pending):
                r = srv.poll(t)
                if r is not None:
                    k = pending.pop(t)
                    lat[k] = time.perf_counter() - t0 - reqs[k][0]
                    done += 1
            if not pending and i < nreq:
                time.sleep(max(0.0, min(0.001, reqs[i][0] - (time.perf_counter() - t0))))
        span = time.perf_counter() - t0
    return lat, span


def serving_measure(pkg, nreq: int, rate: float, tol=None, n_max_exp: float = 5.0,
                    forms=("fp64", "mixed"), gpu: int = 0) -> dict:
    """p50/p99 latency and solves/s of the request stream through the continuous-batching
    server, per served form (request_policy), against the same stream served one request at a
    time by plain FP64 solves of the single-system solver (same shift rule and tolerances).
    tol: one tolerance for every request instead of the trace's own."""
    import numpy as np
    reqs = serving_trace(nreq, rate, n_max_exp=n_max_exp)
    if tol is not None:
        reqs = [(a, P, b, tol) for a, P, b, _ in reqs]
    tol_text = "tol log-uniform [1e-10, 1e-6]" if tol is None else f"tol {tol:g} for every request"
    out = {"workload": f"{nreq} requests, Poisson arrivals {rate:g}/s, n log-uniform [1e3, 1e{n_max_exp:g}], half 2D/3D "
                       f"Laplacian stencils, half random SDD CSR (7-27 nnz/row), {tol_text}",
           "unknowns_total": int(sum(P.n for _, P, _, _ in reqs)),
           "policy": "served_mixed: mixed precision + FP64 refinement; M = I on the Laplacian stencils, Jacobi on "
                     "CSR; served_mixed_jacobi: Jacobi on every request"}

    def summary(lat, span):
        return {"solves_per_s": nreq / span, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "span_s": span}

    for form in forms:
        with ClockSampler(gpu) as clk:
            out[f"served_{form}"] = summary(*serve_stream(pkg, reqs, form))
        out[f"served_{form}"]["clocks"] = clk.summary()
    # one at a time: each request starts when it has arrived and the previous one is done
    # (the shifts are computed before the clock starts)
    sigmas = [request_sigma(P) for _, P, _, _ in reqs]
    lat1 = np.zeros(nreq)
    import gc
    gc.collect()
    gc.disable()
    try:
        with ClockSampler(gpu) as clk:
            t0 = time.perf_counter()
            for k, (arr, P, b, tol) in enumerate(reqs):
                now = time.perf_counter() - t0
                if now < arr:
                    time.sleep(arr - now)
                with pkg.Solver(P) as one:
                    one.solve(b, method="spcg", sigma=sigmas[k], tol=tol, maxit=100000)
                lat1[k] = time.perf_counter() - t0 - arr
            span1 = time.perf_counter() - t0
    finally:
        gc.enable()
    out["one_at_a_time_fp64"] = summary(lat1, span1)
    out["one_at_a_time_fp64"]["clocks"] = clk.summary()
    base = out["one_at_a_time_fp64"]
    for form in forms:
        f = out[f"served_{form}"]
        f["vs_one_at_a_time_fp64"] = {"solves_per_s_ratio": f["solves_per_s"] / base["solves_per_s"],
                                      "p99_ratio": f["p99_ms"] / base["p99_ms"]}
    return out


def request_sigma(P) -> float:
    """The one-at-a-time shift rule: the constant stencil's diagonal, the mean CSR diagonal."""
    import numpy as np
    if P.layout == 0:
        return 4.0
    if P.layout == 1:
        return 6.0
    return float(np.mean(P.val[P.col == np.repeat(np.arange(P.n), np.diff(P.row_ptr))]))


def cpu_side_baselines(S, args, batch, varcoef) -> dict:
    """The oracle (single-threaded FP64, as it stands) beside the side measurements, each on a
    bounded sample scaled to that measurement's unit."""
    import numpy as np
    import oracle
    oracle.build()
    out = {}
    if batch is not None and "fp64_jacobi" in batch:
        # seconds per unknown-iteration of Jacobi shifted p-CG on 4 systems of the batch, times the
        # unknown-iterations the batched FP64 Jacobi solve ran (sum over systems of n x iterations)
        rng = np.random.default_rng(0)
        sides = rng.integers(32, args.batch_side_max + 1, size=args.batch_systems)
        idx = np.linspace(0, args.batch_systems - 1, 4).astype(int)
        k, work, t = 200, 0.0, 0.0
        for i in idx:
            P = S.varcoef_2d(int(sides[i]), int(sides[i]), seed=int(i))
            b = S.normal(1000 + int(i), P.n)
            minv = 1.0 / np.asarray(P.diag)
            t0 = time.perf_counter()
            oracle.pcg_sh(P, b, sigma=1.0, maxit=k, minv=minv, log_every=0)
            t += time.perf_counter() - t0
            work += k * P.n
        est = batch["fp64_jacobi"]["unknown_iterations"] * t / work
        out["batch_fp64_jacobi"] = {
            "solves_per_s": args.batch_systems / est, "est_batch_s": est,
            "sample": f"{k} iterations of 4 of the batch's systems ({t:.1f} s), scaled by the unknown-iterations "
                      "of the batched FP64 Jacobi solve"}
    if varcoef is not None:
        P = S.varcoef_3d(128, block=8, seed=0)
        b = S.normal(1, P.n)
        minv = 1.0 / np.asarray(P.diag)
        k = 30
        t0 = time.perf_counter()
        oracle.pcg_sh(P, b, sigma=varcoef["sigma"], maxit=k, minv=minv, log_every=0)
        t = time.perf_counter() - t0
        out["varcoef_128_fp64_jacobi"] = {
            "iters_per_s": k / t, "est_solve_ms": 1e3 * varcoef["fp64"]["iters"] * t / k,
            "sample": f"{k} iterations of the FP64 Jacobi solve ({t:.1f} s)"}
    if not args.no_serving:
        # the n <= 1e5 stream (a request of the full range alone can keep one core busy for
        # many minutes)
        reqs = serving_trace(max(args.serving_small_requests, 64), args.serving_rate, n_max_exp=5.0, first=64)
        sigmas = [request_sigma(P) for _, P, _, _ in reqs]          # (before the clock starts)
        budget, cnt, t0 = 5.0, 0, time.perf_counter()
        for (_, P, b, tol), sigma in zip(reqs, sigmas):
            oracle.pcg_sh(P, b, sigma=sigma, rtol=tol, maxit=100000, log_every=0)
            cnt += 1
            if time.perf_counter() - t0 > budget:
                break
        t = time.perf_counter() - t0
        out["serving_n_le_1e5_fp64"] = {"solves_per_s": cnt / t,
                                        "sample": f"the n <= 1e5 stream's first {cnt} requests back to back "
                                                  f"({t:.1f} s), FP64, the one-at-a-time shift rule and tolerances"}
    return out


def run_reference(args):
    """The oracle, as it stands, on the host: bounded samples of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import synthetic as S
    P, b, _ = S.poisson3d_manufactured(N_SIDE)
    k = args.ref_iters
    for _ in range(args.warmup):
        cpu_oracle_rate(P, b, k)
    times = []
    for _ in range(args.steps):
        times.append(cpu_oracle_rate(P, b, k)[1])
    total = sum(times)
    value = args.steps * k / total
    sample = (f"{k} iterations of the {N_SIDE}^3 shifted p-CG solve per step (setup of r0, w0 included), "
              "single-threaded FP64 oracle")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(P.n),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


def run_sharded(args, rank: int, world: int, local: int) -> int:
    """One system split over the ranks (weak scaling): the 256 x 256 x (256 N) Laplacian,
    a 256^3 z-slab per GPU, the phases of Algorithm 3 with NCCL halo exchanges and one
    2-scalar all-reduce per iteration (sharded.solve_rank).  `value` is in 256^3
    slab-iterations per second summed over the ranks, the unit of the single-GPU line."""
    import torch
    import synthetic as S
    from paper_1706_05988_gb300 import sharded as SH
    nx = ny = N_SIDE
    nz = N_SIDE * world
    k0, k1 = SH.z_slabs(nz, world)[rank]
    b_local = S.poisson3d_manufactured_slab(nx, ny, nz, k0, k1)
    slab = SH.CudaSlab(nx, ny, k0, k1, nz, b_local, ITERS_PER_STEP)
    comm = SH.DistComm(rank, world)

    def step():
        return SH.solve_rank(slab, comm, SIGMA, 0.0, ITERS_PER_STEP, check_every=0)

    for _ in range(args.warmup):
        res = step()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            res = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    ms_max = max_over_ranks(world, ev0.elapsed_time(ev1))
    value = job_throughput(ITERS_PER_STEP * args.steps, world, ms_max)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"one 7-point Laplacian of {nx}x{ny}x{nz} (x* dyadic U[-1,1] seed 0, b = A x*, "
                                       f"x0 = 0) in {world} z-slabs of {N_SIDE}^3, shifted p-CG sigma={SIGMA}, "
                                       f"{ITERS_PER_STEP} iterations per step; value in {N_SIDE}^3 slab-iterations/s",
                           "n_global": nx * ny * nz, "parallelism": f"z-slabs x{world}",
                           "l2_flush": "not needed: the slab's vectors exceed L2"},
                "sharded": {"iters_per_s_global_system": ITERS_PER_STEP * args.steps / (ms_max / 1e3),
                            "final_true_relres": res["true_relres"], "iters": res["iters"]},
                "e2e": None, "gpu_launches": None, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    slab.close()
    import torch.distributed as dist
    dist.destroy_process_group()
    return 0


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    if args.sharded and world > 1:
        import paper_1706_05988_gb300 as pkg
        if local == 0:
            pkg.build.build()
        barrier(world)
        if local != 0:
            pkg.build.build()
        return run_sharded(args, rank, world, local)
    import paper_1706_05988_gb300 as pkg
    from paper_1706_05988_gb300 import pcg as C
    import synthetic as S

    # one rank builds the in-tree library (a no-op when it is current); the others wait for it
    if local == 0:
        pkg.build.build()
    barrier(world)
    if local != 0:
        pkg.build.build()
    P, b_host, _ = S.poisson3d_manufactured(N_SIDE)
    n = P.n
    solver = pkg.Solver(P, flags=C.PCG_PROFILE)
    stream = torch.cuda.current_stream()
    C.pcg_set_stream(solver.ctx, stream.cuda_stream)
    b_dev = torch.from_numpy(b_host).cuda()
    x_dev = torch.empty(n, dtype=torch.float64, device="cuda")

    def step_device():
        s = C.pcg_solve_device(solver.ctx, b_dev, None, C.PCG_SPCG, SIGMA, 0.0, ITERS_PER_STEP, C.PCG_FP64, x_dev,
                               None)
        if s != C.PCG_ENOTCONV:
            raise C.PcgError(s, C.pcg_last_error(solver.ctx))

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()
    C.pcg_kernel_stats_reset(solver.ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step_device()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    ms = ev0.elapsed_time(ev1)
    launches, iter_launches, iter_ms = C.pcg_kernel_stats(solver.ctx)
    ms_max = max_over_ranks(world, ms)
    total_iters = world * args.steps * ITERS_PER_STEP
    value = job_throughput(args.steps * ITERS_PER_STEP, world, ms_max)

    # roofline of the dominant kernel (the fused iteration), from its own CUDA events
    avg_launch_s = iter_ms / max(iter_launches, 1) / 1e3
    alg_bytes = BYTES_PER_DOF * n
    achieved = alg_bytes / avg_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    sha = kernel_source_sha()
    traffic = NCU_TRAFFIC.get(sha)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": peak_kind, "kernel": "k_spcg_iter (fused SpMV + recurrences + dots)",
                "kernel_avg_ms": avg_launch_s * 1e3, "algorithmic_bytes_per_launch": alg_bytes,
                "kernel_source_sha": sha}
    fp64_tflops = FP64_OPS_PER_DOF * n / avg_launch_s / 1e12

    # end to end: host buffers through pcg_solve (pinned), copies inside the timed region
    b_pin = torch.from_numpy(b_host).pin_memory()
    x_pin = torch.empty(n, dtype=torch.float64).pin_memory()
    res = C.pcg_result()

    def step_host():
        s = C.pcg_solve(solver.ctx, b_pin.data_ptr(), None, C.PCG_SPCG, SIGMA, 0.0, ITERS_PER_STEP, C.PCG_FP64,
                        x_pin.data_ptr(), res)
        if s != C.PCG_ENOTCONV:
            raise C.PcgError(s, C.pcg_last_error(solver.ctx))

    step_host()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_host()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)
    e2e = {"value": total_iters / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
           "final_true_relres": res.final_true_relres}

    # the oracle on this host, bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, dt = cpu_oracle_rate(P, b_host, args.ref_iters)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{args.ref_iters} iterations of the same {N_SIDE}^3 shifted p-CG solve, single-threaded "
                         f"FP64 oracle ({dt:.1f} s; the host has {os.cpu_count()} cores)"}
        # the same source built with OpenMP on its vector loops, on every host core
        try:
            import oracle
            k_omp = 4 * args.ref_iters
            rate_omp, dt_omp = cpu_oracle_rate(P, b_host, k_omp, omp=True)
            cpu["openmp"] = {"value": rate_omp, "unit": UNIT, "cores": oracle.threads(0),
                             "nproc": os.cpu_count(), "speedup_vs_one_core": rate_omp / rate,
                             "sample": f"{k_omp} iterations of the same solve, the oracle's source built with "
                                       f"-fopenmp ({dt_omp:.1f} s)"}
        except Exception as e:   # no OpenMP runtime on this host
            cpu["openmp"] = {"unavailable": str(e)[:200]}

    solver.close()

    # the same step with the persistent cooperative kernel (one launch for all iterations)
    persistent = None
    if not args.no_persistent and world == 1:   # side measurements: single-GPU runs only
        with pkg.Solver(P, flags=C.PCG_PROFILE | C.PCG_PERSISTENT) as sp:
            C.pcg_set_stream(sp.ctx, stream.cuda_stream)
            for _ in range(2):
                s = C.pcg_solve_device(sp.ctx, b_dev, None, C.PCG_SPCG, SIGMA, 0.0, ITERS_PER_STEP, C.PCG_FP64,
                                       x_dev, None)
                assert s == C.PCG_ENOTCONV, C.pcg_last_error(sp.ctx)
            C.pcg_kernel_stats_reset(sp.ctx)
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(args.steps):
                s = C.pcg_solve_device(sp.ctx, b_dev, None, C.PCG_SPCG, SIGMA, 0.0, ITERS_PER_STEP, C.PCG_FP64,
                                       x_dev, None)
            ev1.record(stream)
            torch.cuda.synchronize()
            assert s == C.PCG_ENOTCONV
            _, il, ims = C.pcg_kernel_stats(sp.ctx)
            k_s = ims / il / 1e3                   # per iteration inside the launch
            persistent = {"value": args.steps * ITERS_PER_STEP / (ev0.elapsed_time(ev1) / 1e3), "unit": UNIT,
                          "ms_per_iteration": k_s * 1e3, "achieved_gbs": alg_bytes / k_s / 1e9,
                          "frac": alg_bytes / k_s / 1e9 / peak}

    # batch of independent 2D variable-coefficient systems in one persistent launch vs one at a time
    batch = None
    if not args.no_batch and world == 1:   # side measurements: single-GPU runs only
        batch = batch_measure(pkg, S, args.batch_systems, args.batch_side_max, peak_gbs=peak)

    varcoef = None
    if not args.no_varcoef and world == 1:   # side measurements: single-GPU runs only
        varcoef = varcoef_measure(pkg, S)

    serving = serving_1e8 = serving_small = serving_small_1e8 = None
    if not args.no_serving and world == 1:   # side measurements: single-GPU runs only
        # the serving workload's full size range, on a bounded number of requests
        serving_1e8 = serving_measure(pkg, args.serving_requests, args.serving_rate, tol=1e-8,
                                      n_max_exp=args.serving_n_max_exp, gpu=local)
        serving = serving_measure(pkg, args.serving_requests, args.serving_rate, n_max_exp=args.serving_n_max_exp,
                                  gpu=local)
        # many small requests: n up to 1e5, where the cluster lanes carry everything
        if args.serving_small_requests > 0:
            small = ("fp64", "mixed", "mixed_jacobi")
            serving_small_1e8 = serving_measure(pkg, args.serving_small_requests, args.serving_rate, tol=1e-8,
                                                n_max_exp=5.0, forms=small, gpu=local)
            serving_small = serving_measure(pkg, args.serving_small_requests, args.serving_rate, n_max_exp=5.0,
                                            forms=small, gpu=local)

    # the same workload as CSR (int32 indices): config's second form, one timed step
    csr = None
    if not args.no_csr and world == 1:   # side measurements: single-GPU runs only
        Pc = S.to_csr(P)
        bytes_csr = BYTES_PER_DOF * n + 12 * Pc.nnz + 4 * (n + 1)
        with pkg.Solver(Pc, flags=C.PCG_PROFILE) as sc:
            C.pcg_set_stream(sc.ctx, stream.cuda_stream)
            for _ in range(2):
                s = C.pcg_solve_device(sc.ctx, b_dev, None, C.PCG_SPCG, SIGMA, 0.0, ITERS_PER_STEP, C.PCG_FP64,
                                       x_dev, None)
                assert s == C.PCG_ENOTCONV, C.pcg_last_error(sc.ctx)
            C.pcg_kernel_stats_reset(sc.ctx)
            torch.cuda.synchronize()
            ev0.record(stream)
            s = C.pcg_solve_device(sc.ctx, b_dev, None, C.PCG_SPCG, SIGMA, 0.0, ITERS_PER_STEP, C.PCG_FP64, x_dev, None)
            ev1.record(stream)
            torch.cuda.synchronize()
            assert s == C.PCG_ENOTCONV
            _, il, ims = C.pcg_kernel_stats(sc.ctx)
            k_s = ims / il / 1e3
            csr = {"value": ITERS_PER_STEP / (ev0.elapsed_time(ev1) / 1e3), "unit": UNIT, "nnz": Pc.nnz,
                   "kernel_avg_ms": k_s * 1e3, "algorithmic_bytes_per_launch": bytes_csr,
                   "achieved_gbs": bytes_csr / k_s / 1e9, "frac": bytes_csr / k_s / 1e9 / peak}
        del Pc

    if cpu is not None:
        cpu["side"] = cpu_side_baselines(S, args, batch, varcoef)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(n),
                "hbm_gbs_effective": alg_bytes * ITERS_PER_STEP * args.steps * world / (ms_max / 1e3) / 1e9 / world,
                "roofline": roofline,
                "fp64_pipe": {"achieved_tinst_per_s": fp64_tflops, "ops_per_dof": FP64_OPS_PER_DOF,
                              "peak_tinst_per_s": 2 * 152 * 2.07e9 / 1e12,
                              "note": "FP64 thread-instructions per unknown per iteration; peak = 2 per cycle "
                                      "per SM x 152 SMs x 2.07 GHz (ncu sm__sass_thread_inst_executed_op_dfma "
                                      "peak_sustained)"},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary(),
                "csr_int32": csr, "persistent": persistent, "varcoef_128": varcoef, "batch": batch,
                "serving": serving, "serving_tol_1e-8": serving_1e8,
                "serving_n_le_1e5": serving_small, "serving_n_le_1e5_tol_1e-8": serving_small_1e8}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def profile_case(kind: str, n: int) -> int:
    """A short solve for an ncu capture (no timing, no JSON): `spcg` runs 8 iterations of the
    main kernel on the n^3 Laplacian (`spcg2d`: on the n^2 Laplacian, `spcg2d-mixed`: its mixed-precision
    sweep for 12 iterations with eta = 1e-30; `-split32`: with the dots on the FP32 pipe; `-staged`: the
    TMA-staged sweep with a ring of 2 chunks); `jacobi-fp64` and `jacobi-mixed` run 12 iterations of the
    Jacobi sweeps (sigma = 1; the mixed one with eta = 1e-30, so no restart interrupts);
    `batch-*` run batched launches (see below)."""
    import synthetic as S
    import paper_1706_05988_gb300 as pkg
    from paper_1706_05988_gb300 import pcg as C
    pkg.build.build()
    if kind.startswith("batch-large"):
        # one batched launch of the large systems of the 512-system batch: 64 2D FV systems with
        # sides U{256..512} (9.6M unknowns), 500 iterations each, Jacobi, cluster size 2
        import numpy as np
        rng = np.random.default_rng(0)
        probs = [S.varcoef_2d(int(L), int(L), seed=i) for i, L in enumerate(rng.integers(256, 513, size=64))]
        bs = [S.normal(1000 + i, P.n) for i, P in enumerate(probs)]
        prec = C.PCG_MIXED_IR if kind.startswith("batch-large-mixed-jacobi") else C.PCG_FP64
        with pkg.Batch(probs, flags=pkg.PCG_JACOBI, precision=prec) as bt:
            # cluster size 2 (the shape the autotuner takes for the large class of the
            # 512-system batch); -c16: 16 blocks per system and the 4-block variant, the
            # fastest shape for these 64 systems alone
            bt.set_cluster(16 if kind.endswith("-c16") else 2)
            if kind.endswith("-occ4") or kind.endswith("-c16"):
                bt.set_class_occupancy(2, 4)      # the 64-register kernel variant, forced
            for _ in range(2):
                _, it, st, _ = bt.solve(bs, [1.0] * len(probs), tol=1e-8, maxit=500)
            print(kind, "kernel ms", bt.last_kernel_ms(), "unknowns", sum(P.n for P in probs), "iterations", int(it.max()))
        return 0
    if kind.startswith("batch"):
        # one batched launch: 128 2D FV systems (sides U{32..128}) to 1e-8, cluster size 4
        import numpy as np
        rng = np.random.default_rng(0)
        probs = [S.varcoef_2d(int(L), int(L), seed=i) for i, L in enumerate(rng.integers(32, 129, size=128))]
        bs = [S.normal(1000 + i, P.n) for i, P in enumerate(probs)]
        jac = kind == "batch-mixed-jacobi"
        sig = [1.0] * len(probs) if jac else [0.5 * float(np.median(P.diag)) for P in probs]
        with pkg.Batch(probs, flags=pkg.PCG_JACOBI if jac else 0,
                       precision=C.PCG_MIXED_IR if jac else C.PCG_FP64) as bt:
            bt.set_cluster(4)
            for _ in range(2):
                _, it, st, _ = bt.solve(bs, sig, tol=1e-8, maxit=100000)
        print(kind, int(np.sum(st == 0)), float(np.mean(it)))
        return 0
    if kind in ("spcg2d", "spcg2d-mixed"):
        P = S.laplacian_2d(n)
        with pkg.Solver(P) as s:
            if kind == "spcg2d":
                r = s.solve(S.normal(0, P.n), method="spcg", sigma=4.0, maxit=8)
            else:
                C.pcg_set_param(s.ctx, C.PCG_PARAM_MIXED_ETA, 1e-30)
                r = s.solve(S.normal(0, P.n), method="spcg", sigma=4.0, maxit=12, precision=C.PCG_MIXED_IR)
        print(kind, n, r.status, r.iters)
        return 0
    P, b = S.poisson3d_manufactured(n)[:2]
    if kind.startswith("spcg"):
        with pkg.Solver(P, flags=pkg.PCG_DOTS_SPLIT32 if "split32" in kind else 0) as s:
            if "staged" in kind:
                C.pcg_set_param(s.ctx, C.PCG_PARAM_ITER_STAGES, 2.0)
            r = s.solve(b, method="spcg", sigma=6.0, maxit=8)
    else:
        with pkg.Solver(P, flags=pkg.PCG_JACOBI) as s:
            if kind == "jacobi-fp64":
                r = s.solve(b, method="spcg", sigma=1.0, maxit=12)
            else:
                C.pcg_set_param(s.ctx, C.PCG_PARAM_MIXED_ETA, 1e-30)
                r = s.solve(b, method="spcg", sigma=1.0, maxit=12, precision=C.PCG_MIXED_IR)
    print(kind, n, r.status, r.iters)
    return 0


def compare_iter_forms(n: int) -> int:
    """Event-timed A/B of the forms of the fused iteration on the n^3 Laplacian (1,000
    iterations each, best of 3): the register sweep and the TMA-staged sweep (rings of 2
    and 3 chunks), each with binary64 dots and with the dots on the FP32 pipe; prints one
    JSON line of kernel ms per launch and algorithmic GB/s (96 B per unknown)."""
    import torch
    import synthetic as S
    import paper_1706_05988_gb300 as pkg
    from paper_1706_05988_gb300 import pcg as C
    pkg.build.build()
    P, b, _ = S.poisson3d_manufactured(n)
    bd = torch.from_numpy(b).cuda()
    out = {"workload": f"{n}^3 Laplacian, shifted p-CG sigma={SIGMA}, 1000 iterations"}
    for dots, fl in (("fp64_dots", 0), ("split32_dots", C.PCG_DOTS_SPLIT32)):
        with pkg.Solver(P, flags=C.PCG_PROFILE | fl) as s:
            for stages in (0, 2, 3):
                C.pcg_set_param(s.ctx, C.PCG_PARAM_ITER_STAGES, float(stages))
                got = int(C.pcg_get_param(s.ctx, C.PCG_PARAM_ITER_STAGES))
                s.solve(bd, method="spcg", sigma=SIGMA, maxit=50, device=True)
                best = None
                for _ in range(3):
                    C.pcg_kernel_stats_reset(s.ctx)
                    s.solve(bd, method="spcg", sigma=SIGMA, maxit=1000, device=True)
                    _, il, ims = C.pcg_kernel_stats(s.ctx)
                    best = ims / il if best is None else min(best, ims / il)
                key = f"{'register' if got == 0 else f'staged{got}'}_{dots}"
                out[key] = {"kernel_ms": best, "algorithmic_gbs": BYTES_PER_DOF * P.n / best / 1e6}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile-case", choices=["spcg", "spcg2d", "spcg2d-mixed", "spcg-split32", "spcg-staged", "spcg-staged-split32",
                                               "jacobi-fp64", "jacobi-mixed", "batch-fp64",
                                               "batch-mixed-jacobi", "batch-large-fp64-jacobi",
                                               "batch-large-mixed-jacobi", "batch-large-mixed-jacobi-occ4", "batch-large-mixed-jacobi-c16",
                                               "batch-large-fp64-jacobi-c16"],
                    default=None,
                    help="run one short solve of --size^3 for an ncu capture, then exit")
    ap.add_argument("--compare-iter-forms", action="store_true",
                    help="time the register and TMA-staged sweeps with both dot forms on --size^3, then exit")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--sharded", action="store_true",
                    help="with N > 1 GPUs: one 256x256x(256N) system in z-slabs (halo exchange and an all-reduce "
                         "per iteration) instead of N independent 256^3 systems")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-iters", type=int, default=50, help="oracle iterations per sample (about 11 s on one core)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle timing")
    ap.add_argument("--no-csr", action="store_true", help="skip the CSR form of the workload")
    ap.add_argument("--no-persistent", action="store_true", help="skip the persistent-kernel measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-solve measurement")
    ap.add_argument("--no-varcoef", action="store_true", help="skip the 128^3 variable-coefficient measurement")
    ap.add_argument("--batch-systems", type=int, default=512, help="systems in the batched-solve measurement")
    ap.add_argument("--batch-side-max", type=int, default=512, help="batched systems have sides U{32..this}")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serving-requests", type=int, default=48,
                    help="requests of the full-range serving stream (n log-uniform in [1e3, 1e7])")
    ap.add_argument("--serving-small-requests", type=int, default=400,
                    help="requests of the extra serving stream with n <= 1e5 (0: skip it)")
    ap.add_argument("--serving-rate", type=float, default=2000.0, help="Poisson arrival rate, requests/s")
    ap.add_argument("--serving-n-max-exp", type=float, default=7.0,
                    help="serving requests have n log-uniform in [1e3, 10^this] (the serving workload's range: 7)")
    ap.add_argument("--size", type=int, default=N_SIDE, help="grid side (default: the 256^3 workload)")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args.profile_case, args.size)
    if args.compare_iter_forms:
        return compare_iter_forms(args.size)
    globals()["N_SIDE"] = args.size
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

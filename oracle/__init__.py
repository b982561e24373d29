"""Oracle for the shifted pipelined CG hot path (arXiv 1706.05988).

TEST INFRASTRUCTURE ONLY: a plain, slow, single-threaded FP64 CPU
implementation used to check the CUDA path.  Only tests/,
__graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may
import it.  It shares no code with the CUDA path; the only module both sides
use is `synthetic` (seeded problem data, none of the solver's arithmetic).

Contents
  build()          compile pcg_oracle.c with gcc (-O2 -ffp-contract=off); build(omp=True)
                   also with -fopenmp, a second library used only to time the oracle on
                   every host core (threads() sets its thread count)
  apply(P, x)      y = A x                         (operator of the model problem)
  cg(...)          Algorithm 1, classic CG
  pcg(...)         Algorithm 2, pipelined CG (written out without shift terms)
  pcg_varsh(...)   Algorithm 4, pipelined CG with a variable shift
  pcg_sh(...)      Algorithm 3, shifted pipelined CG
  psi / select_sigma   Section 3.2, Eq. (functionpsi)        -> oracle.psi
  exact rational CG / p-CG-sh for tiny systems               -> oracle.exact

Every function above is pinned by tests/test_oracle.py (exact arithmetic, closed forms,
library routines, the values Table 1 and Section 5.1 print).  Parity unpinned: the level
at which unshifted p-CG (Algorithm 2) stalls on lapl200, which Table 1 prints as 3.1e-7.
It depends on rounding after the iteration has lost its way; only its order relative to
CG (at least 100 times higher) is tested.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lib = None
_lib_omp = None

OP_CSR, OP_STENCIL2D, OP_STENCIL3D = 0, 1, 2


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle shared library (plain C, no vectorisation tricks; single-threaded).
    omp=True: the same source built a second time with -fopenmp (its vector loops and
    reductions on all host cores), for timing only -- its reductions sum in another order,
    and nothing compares against it."""
    os.makedirs(_BUILD, exist_ok=True)
    lib = _LIB_OMP if omp else _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               *(["-fopenmp"] if omp else []), "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, lib)
    return lib


class _Op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int64), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("nz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("diag", ctypes.c_void_p), ("ax", ctypes.c_void_p),
                ("ay", ctypes.c_void_p), ("az", ctypes.c_void_p)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32)]


class _State(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("x", "r", "u", "w", "z", "q", "s", "t", "p")]


def _declare(lib):
    vp, i32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    lib.oracle_apply.argtypes = [vp, vp, vp]
    lib.oracle_cg.argtypes = [vp, vp, vp, vp, i32, f64, f64, i32, vp, vp, vp, vp, vp, vp]
    lib.oracle_pcg_sh.argtypes = [vp, vp, vp, vp, f64, i32, f64, f64, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                  vp, vp, vp]
    lib.oracle_pcg.argtypes = [vp, vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.oracle_pcg_varsh.argtypes = [vp, vp, vp, vp, vp, i32, f64, i32, vp, vp, vp, vp, vp, vp]
    lib.oracle_threads.argtypes = [i32]
    for f in (lib.oracle_cg, lib.oracle_pcg_sh, lib.oracle_pcg, lib.oracle_pcg_varsh, lib.oracle_threads):
        f.restype = ctypes.c_int
    return lib


def threads(n: int = 0, omp: bool = True) -> int:
    """Set (n > 0) and return the thread count of the OpenMP build (1 for the serial one)."""
    return _load(omp).oracle_threads(n)


def _load(omp: bool = False):
    global _lib, _lib_omp
    if omp:
        if _lib_omp is None:
            _lib_omp = _declare(ctypes.CDLL(build(omp=True)))
        return _lib_omp
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


class _OpHolder:
    """Keeps the numpy arrays referenced by the C struct alive."""

    def __init__(self, P):
        from synthetic import CSR32, STENCIL5_2D
        self.keep = []

        def c(a, dt):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dt)
            self.keep.append(a)
            return a.ctypes.data

        op = _Op()
        if P.layout == CSR32:
            op.kind, op.n = OP_CSR, P.n
            op.row_ptr, op.col, op.val = c(P.row_ptr, np.int32), c(P.col, np.int32), c(P.val, np.float64)
        else:
            op.kind = OP_STENCIL2D if P.layout == STENCIL5_2D else OP_STENCIL3D
            op.n, op.nx, op.ny, op.nz = P.n, P.nx, P.ny, P.nz
            if not P.constant:
                op.diag, op.ax, op.ay, op.az = (c(P.diag, np.float64), c(P.ax, np.float64),
                                                c(P.ay, np.float64), c(P.az, np.float64))
        self.op = op

    @property
    def ref(self):
        return ctypes.byref(self.op)


@dataclass
class Run:
    """Output of one oracle solve.  Histories have length iters+1 (alpha/beta: iters)."""
    x: np.ndarray
    iters: int
    status: int            # 0 maxit, 1 converged, 2 breakdown
    alpha: np.ndarray
    beta: np.ndarray
    rec: np.ndarray        # ||r_i||
    true: np.ndarray       # ||b - A x_i|| (NaN where not logged)
    gap: np.ndarray        # ||(b - A x_i) - r_i||
    gamma: Optional[np.ndarray] = None
    delta: Optional[np.ndarray] = None
    state: Optional[dict] = None
    gap_g: Optional[np.ndarray] = None     # ||(A p_i - sigma t_i) - s_i||   (Section 3.1; NaN where not logged)
    gap_h: Optional[np.ndarray] = None     # ||(A u_i - sigma r_i) - w_i||
    gap_j: Optional[np.ndarray] = None     # ||A q_i - z_i||


def apply(P, x: np.ndarray) -> np.ndarray:
    """y = A x with the oracle's own operator code."""
    lib = _load()
    h = _OpHolder(P)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    lib.oracle_apply(h.ref, x.ctypes.data, y.ctypes.data)
    return y


def _hist(maxit):
    return [np.full(maxit + 1, np.nan) for _ in range(5)]


def _minv(minv):
    return None if minv is None else np.ascontiguousarray(minv, dtype=np.float64)


def cg(P, b, x0=None, maxit=100, rtol=0.0, ttol=0.0, log_every=1, minv=None) -> Run:
    """Algorithm 1 (classic preconditioned CG)."""
    lib = _load()
    h = _OpHolder(P)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(P.n) if x0 is None else np.array(x0, dtype=np.float64)
    al, be, rec, tru, gap = _hist(maxit)
    info = _Info()
    mv = _minv(minv)
    rc = lib.oracle_cg(h.ref, _ptr(mv), b.ctypes.data, x.ctypes.data, maxit, rtol, ttol, log_every,
                       al.ctypes.data, be.ctypes.data, rec.ctypes.data, tru.ctypes.data, gap.ctypes.data,
                       ctypes.byref(info))
    if rc != 0:
        raise MemoryError("oracle_cg allocation failed")
    k = info.iters
    return Run(x, k, info.status, al[:k], be[:k], rec[:k + 1], tru[:k + 1], gap[:k + 1])


def pcg_sh(P, b, x0=None, sigma=0.0, maxit=100, rtol=0.0, ttol=0.0, log_every=1, minv=None,
           want_state=False, omp=False, gaps=False) -> Run:
    """Algorithm 3 (shifted pipelined CG); sigma = 0 gives Algorithm 2's recurrences.
    gaps=True also logs ||g_i||, ||h_i||, ||j_i|| (Section 3.1) where the true residual is
    logged.  omp=True runs the OpenMP build (timing only; see build)."""
    lib = _load(omp)
    h = _OpHolder(P)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(P.n) if x0 is None else np.array(x0, dtype=np.float64)
    al, be, rec, tru, gap = _hist(maxit)
    ga = np.full(maxit + 1, np.nan)
    de = np.full(maxit + 1, np.nan)
    info = _Info()
    st = None
    stp = None
    if want_state:
        st = {k: np.zeros(P.n) for k in ("x", "r", "u", "w", "z", "q", "s", "t", "p")}
        cs = _State(**{k: v.ctypes.data for k, v in st.items()})
        stp = ctypes.byref(cs)
    mv = _minv(minv)
    gg, hh, jj = (np.full(maxit + 1, np.nan) for _ in range(3))
    want = gaps and log_every > 0
    rc = lib.oracle_pcg_sh(h.ref, _ptr(mv), b.ctypes.data, x.ctypes.data, float(sigma), maxit, rtol, ttol,
                           log_every, al.ctypes.data, be.ctypes.data, rec.ctypes.data, tru.ctypes.data,
                           gap.ctypes.data, ga.ctypes.data, de.ctypes.data, ctypes.byref(info), stp,
                           gg.ctypes.data if want else None, hh.ctypes.data if want else None,
                           jj.ctypes.data if want else None)
    if rc != 0:
        raise MemoryError("oracle_pcg_sh allocation failed")
    k = info.iters
    return Run(x, k, info.status, al[:k], be[:k], rec[:k + 1], tru[:k + 1], gap[:k + 1], ga[:k], de[:k], st,
               gg[:k + 1] if want else None, hh[:k + 1] if want else None, jj[:k + 1] if want else None)


def pcg(P, b, x0=None, maxit=100, log_every=1, minv=None) -> Run:
    """Algorithm 2 (pipelined CG), the separate unshifted code path."""
    lib = _load()
    h = _OpHolder(P)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(P.n) if x0 is None else np.array(x0, dtype=np.float64)
    al, be, rec, tru, gap = _hist(maxit)
    info = _Info()
    mv = _minv(minv)
    rc = lib.oracle_pcg(h.ref, _ptr(mv), b.ctypes.data, x.ctypes.data, maxit, log_every, al.ctypes.data,
                        be.ctypes.data, rec.ctypes.data, tru.ctypes.data, gap.ctypes.data, ctypes.byref(info))
    if rc != 0:
        raise MemoryError("oracle_pcg allocation failed")
    k = info.iters
    return Run(x, k, info.status, al[:k], be[:k], rec[:k + 1], tru[:k + 1], gap[:k + 1])


def pcg_varsh(P, b, shifts, x0=None, maxit=100, rtol=0.0, log_every=1, minv=None) -> Run:
    """Algorithm 4: shifts[0] = sigma_{-1}, shifts[k + 1] = sigma_k (at least maxit + 1 values)."""
    lib = _load()
    h = _OpHolder(P)
    b = np.ascontiguousarray(b, dtype=np.float64)
    sh = np.ascontiguousarray(shifts, dtype=np.float64)
    if sh.size < maxit + 1:
        raise ValueError("need maxit + 1 shifts")
    x = np.zeros(P.n) if x0 is None else np.array(x0, dtype=np.float64)
    al, be, rec, tru, gap = _hist(maxit)
    info = _Info()
    mv = _minv(minv)
    rc = lib.oracle_pcg_varsh(h.ref, _ptr(mv), b.ctypes.data, x.ctypes.data, sh.ctypes.data, maxit, rtol, log_every,
                              al.ctypes.data, be.ctypes.data, rec.ctypes.data, tru.ctypes.data, gap.ctypes.data,
                              ctypes.byref(info))
    if rc != 0:
        raise MemoryError("oracle_pcg_varsh allocation failed")
    k = info.iters
    return Run(x, k, info.status, al[:k], be[:k], rec[:k + 1], tru[:k + 1], gap[:k + 1])

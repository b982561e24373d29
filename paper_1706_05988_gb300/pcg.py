"""ctypes binding of libpcg (C ABI in include/pcg.h): argument marshalling only.

Every function named pcg_* here calls the C function of the same name.  The
library must have been built (build.build()); loading fails loudly otherwise,
and there is no fallback path of any kind.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PCG_LIBRARY selects another build of the same C ABI (libpcg_checked.so, the index-checked
# build); it must exist -- there is no fallback of any kind
LIB_PATH = os.environ.get("PCG_LIBRARY") or os.path.join(_HERE, "libpcg.so")

# pcg_status
PCG_OK, PCG_EINVAL, PCG_ENOMEM, PCG_ECUDA, PCG_EBREAKDOWN, PCG_ENOTCONV, PCG_ETIMEOUT, PCG_PENDING, PCG_ENOTIMPL = range(9)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EBREAKDOWN", 5: "ENOTCONV", 6: "ETIMEOUT",
                7: "PENDING", 8: "ENOTIMPL"}
# pcg_layout / pcg_method / pcg_precision
PCG_STENCIL5_2D, PCG_STENCIL7_3D, PCG_CSR32 = 0, 1, 2
PCG_CG, PCG_PCG, PCG_SPCG = 0, 1, 2
PCG_FP64, PCG_MIXED_IR = 0, 1
# pcg_create flags
PCG_DEVICE_PTRS = 0x1
PCG_PROFILE = 0x2
PCG_STENCIL_FP64_SUM = 0x4
# pcg_set_param parameters
PCG_PARAM_MIXED_ETA, PCG_PARAM_MAX_RESTARTS, PCG_PARAM_BARRIER_TIMEOUT_MS, PCG_PARAM_TEST_BARRIER_PHANTOMS = 1, 2, 3, 4
PCG_PARAM_TRUE_TOL = 5
PCG_PARAM_ITER_STAGES = 6
PCG_SCALAR_LOG = 32
PCG_PERSISTENT = 0x8
PCG_JACOBI = 0x10
PCG_DOTS_SPLIT32 = 0x20

METHODS = {"cg": PCG_CG, "pcg": PCG_PCG, "spcg": PCG_SPCG}


class PcgError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        super().__init__(f"pcg status {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class pcg_matrix(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_int32), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("diag", ctypes.c_void_p), ("ax", ctypes.c_void_p), ("ay", ctypes.c_void_p), ("az", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class pcg_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("final_true_relres", ctypes.c_double),
                ("final_rec_relres", ctypes.c_double), ("rec_hist", ctypes.c_void_p),
                ("true_hist", ctypes.c_void_p), ("gap_hist", ctypes.c_void_p), ("alpha_hist", ctypes.c_void_p),
                ("beta_hist", ctypes.c_void_p), ("true_every", ctypes.c_int32)]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libpcg (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{os.path.basename(LIB_PATH)} not found at {LIB_PATH}: run __graft_entry__.build() first "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, f64, st = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        L.pcg_create.argtypes = [ctypes.POINTER(pcg_matrix), ctypes.c_uint32, ctypes.POINTER(vp)]
        L.pcg_destroy.argtypes = [vp]
        L.pcg_destroy.restype = None
        L.pcg_last_error.argtypes = [vp]
        L.pcg_last_error.restype = ctypes.c_char_p
        L.pcg_set_stream.argtypes = [vp, vp]
        solve_args = [vp, vp, vp, i32, f64, f64, i32, i32, vp, ctypes.POINTER(pcg_result)]
        L.pcg_solve.argtypes = solve_args
        L.pcg_solve_device.argtypes = solve_args
        L.pcg_select_sigma.argtypes = [vp, vp, i32, vp, i32, ctypes.POINTER(f64), vp]
        L.pcg_psi.argtypes = [vp, vp, vp, i32, vp, i32, vp]
        L.pcg_apply.argtypes = [vp, vp, vp]
        L.pcg_set_param.argtypes = [vp, i32, f64]
        L.pcg_get_param.argtypes = [vp, i32, ctypes.POINTER(f64)]
        L.pcg_set_shifts.argtypes = [vp, vp, i32]
        L.pcg_psi_varsh.argtypes = [vp, vp, vp, i32, vp, i32, i32, vp]
        L.pcg_batch_create.argtypes = [vp, i32, ctypes.c_uint32, ctypes.POINTER(vp)]
        L.pcg_batch_solve.argtypes = [vp, vp, vp, i32, vp, f64, i32, vp, vp, vp]
        L.pcg_batch_autotune.argtypes = [vp, vp, vp, i32, vp, vp]
        L.pcg_batch_set_cluster.argtypes = [vp, i32]
        L.pcg_batch_set_precision.argtypes = [vp, i32]
        L.pcg_batch_classes.argtypes = [vp, vp, vp, vp]
        L.pcg_batch_set_class_cluster.argtypes = [vp, i32, i32]
        L.pcg_batch_set_class_occupancy.argtypes = [vp, i32, i32]
        L.pcg_batch_set_param.argtypes = [vp, i32, f64]
        L.pcg_batch_last_kernel_ms.argtypes = [vp, ctypes.POINTER(f64)]
        L.pcg_batch_scalars.argtypes = [vp, i32, vp, vp]
        L.pcg_batch_destroy.argtypes = [vp]
        L.pcg_batch_destroy.restype = None
        L.pcg_server_create.argtypes = [ctypes.c_size_t, i32, ctypes.POINTER(vp)]
        L.pcg_submit.argtypes = [vp, ctypes.POINTER(pcg_matrix), vp, f64, i32, f64, i32, ctypes.POINTER(ctypes.c_uint64)]
        L.pcg_submit_ex.argtypes = [vp, ctypes.POINTER(pcg_matrix), vp, f64, i32, f64, i32, ctypes.c_uint32, i32,
                                    ctypes.POINTER(ctypes.c_uint64)]
        L.pcg_poll.argtypes = [vp, ctypes.c_uint64, vp, ctypes.POINTER(pcg_result)]
        L.pcg_server_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_size_t)]
        L.pcg_server_destroy.argtypes = [vp]
        L.pcg_server_destroy.restype = None
        L.pcg_convert_check.argtypes = [vp, vp, vp, vp, i64]
        L.pcg_true_residual_noalloc.argtypes = [ctypes.POINTER(pcg_matrix), vp, vp, vp, vp, vp]
        L.pcg_kernel_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(f64)]
        L.pcg_kernel_stats_reset.argtypes = [vp]
        L.pcg_check_status.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(i32)]
        L.pcg_version.argtypes = []
        L.pcg_version.restype = ctypes.c_char_p
        for f in ("pcg_create", "pcg_set_stream", "pcg_solve", "pcg_solve_device", "pcg_select_sigma", "pcg_psi",
                  "pcg_apply", "pcg_true_residual_noalloc", "pcg_set_param", "pcg_get_param", "pcg_set_shifts", "pcg_convert_check",
                  "pcg_psi_varsh",
                  "pcg_batch_create", "pcg_batch_solve", "pcg_batch_autotune", "pcg_batch_set_cluster",
                  "pcg_batch_set_precision", "pcg_batch_set_param", "pcg_batch_last_kernel_ms", "pcg_batch_scalars",
                  "pcg_server_create",
                  "pcg_batch_classes", "pcg_batch_set_class_cluster", "pcg_batch_set_class_occupancy",
                  "pcg_submit", "pcg_submit_ex", "pcg_poll", "pcg_server_stats",
                  "pcg_kernel_stats", "pcg_kernel_stats_reset", "pcg_check_status"):
            getattr(L, f).restype = st
        _lib = L
    return _lib


def _p(a) -> Optional[int]:
    """Address of a numpy array / torch tensor / int (None stays None)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    raise TypeError(type(a))


# ---------------------------------------------------------------- same-name wrappers

def pcg_version() -> str:
    return lib().pcg_version().decode()


def pcg_last_error(ctx) -> str:
    return lib().pcg_last_error(ctx).decode()


def pcg_create(A: pcg_matrix, flags: int = 0) -> int:
    out = ctypes.c_void_p()
    s = lib().pcg_create(ctypes.byref(A), flags, ctypes.byref(out))
    if s != PCG_OK:
        raise PcgError(s, "pcg_create")
    return out.value


def pcg_destroy(ctx) -> None:
    lib().pcg_destroy(ctx)


def pcg_set_stream(ctx, stream_ptr: int) -> int:
    return lib().pcg_set_stream(ctx, stream_ptr)


def pcg_solve(ctx, b, x0, method, sigma, tol, maxit, precision, x_out, res) -> int:
    return lib().pcg_solve(ctx, _p(b), _p(x0), method, sigma, tol, maxit, precision, _p(x_out),
                           ctypes.byref(res) if res is not None else None)


def pcg_solve_device(ctx, b, x0, method, sigma, tol, maxit, precision, x_out, res) -> int:
    return lib().pcg_solve_device(ctx, _p(b), _p(x0), method, sigma, tol, maxit, precision, _p(x_out),
                                  ctypes.byref(res) if res is not None else None)


def pcg_set_param(ctx, param: int, value: float) -> int:
    return lib().pcg_set_param(ctx, param, value)


def pcg_psi_varsh(ctx, alpha, beta, i: int, schedules) -> np.ndarray:
    """psi_i for each row of `schedules` (2D, one shift schedule per row, >= i + 2 columns)."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    sch = np.ascontiguousarray(np.atleast_2d(schedules), dtype=np.float64)
    out = np.zeros(sch.shape[0])
    s = lib().pcg_psi_varsh(ctx, a.ctypes.data, b.ctypes.data, i, sch.ctypes.data, sch.shape[1], sch.shape[0],
                            out.ctypes.data)
    if s != PCG_OK:
        raise PcgError(s, "pcg_psi_varsh")
    return out


def pcg_set_shifts(ctx, shifts) -> int:
    if shifts is None:
        return lib().pcg_set_shifts(ctx, None, 0)
    a = np.ascontiguousarray(shifts, dtype=np.float64)
    return lib().pcg_set_shifts(ctx, a.ctypes.data, a.size)


def pcg_apply(ctx, x, y) -> int:
    """y = A x on the device (x, y: CUDA tensors or device addresses)."""
    return lib().pcg_apply(ctx, _p(x), _p(y))


def pcg_true_residual_noalloc(A: pcg_matrix, b, x, r, norms, stream=None) -> int:
    """||b - A x|| and ||(b - A x) - r|| into the device array norms[2] without allocating;
    A's arrays, b, x, r (or None) and norms are device memory (tensors or addresses)."""
    return lib().pcg_true_residual_noalloc(ctypes.byref(A), _p(b), _p(x), _p(r), _p(norms), stream)


def pcg_psi(ctx, alpha: np.ndarray, beta: np.ndarray, i: int, grid: np.ndarray) -> np.ndarray:
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    grid = np.ascontiguousarray(grid, dtype=np.float64)
    out = np.empty(grid.size)
    s = lib().pcg_psi(ctx, _p(alpha), _p(beta), i, _p(grid), grid.size, _p(out))
    if s != PCG_OK:
        raise PcgError(s, pcg_last_error(ctx))
    return out


def pcg_select_sigma(ctx, b: np.ndarray, iters: int, grid) -> tuple[float, np.ndarray]:
    b = np.ascontiguousarray(b, dtype=np.float64)
    grid = np.ascontiguousarray(grid, dtype=np.float64)
    sig = ctypes.c_double()
    psi = np.empty(grid.size)
    s = lib().pcg_select_sigma(ctx, _p(b), iters, _p(grid), grid.size, ctypes.byref(sig), _p(psi))
    if s != PCG_OK:
        raise PcgError(s, pcg_last_error(ctx))
    return sig.value, psi


def pcg_get_param(ctx, param: int) -> float:
    v = ctypes.c_double()
    s = lib().pcg_get_param(ctx, param, ctypes.byref(v))
    if s != PCG_OK:
        raise PcgError(s, "pcg_get_param")
    return v.value


def pcg_check_status() -> tuple[int, bool]:
    """(first failed index-check code since the last call or 0, whether this is the checked build)."""
    code, checked = ctypes.c_uint32(), ctypes.c_int32()
    s = lib().pcg_check_status(ctypes.byref(code), ctypes.byref(checked))
    if s != PCG_OK:
        raise PcgError(s, "pcg_check_status")
    return code.value, bool(checked.value)


def pcg_kernel_stats(ctx) -> tuple[int, int, float]:
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    s = lib().pcg_kernel_stats(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    if s != PCG_OK:
        raise PcgError(s)
    return a.value, b.value, c.value


def pcg_kernel_stats_reset(ctx) -> None:
    lib().pcg_kernel_stats_reset(ctx)


# ---------------------------------------------------------------- convenience

class Matrix:
    """pcg_matrix built from a problem description (duck-typed: layout, nx, ny,
    nz, diag/ax/ay/az or row_ptr/col/val), keeping its arrays alive."""

    def __init__(self, P, device_arrays: Optional[dict] = None):
        self.keep = []
        m = pcg_matrix()
        m.layout = P.layout

        def arr(a, dt):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dt)
            self.keep.append(a)
            return a.ctypes.data

        if device_arrays is not None:      # torch tensors on the GPU
            self.keep.append(device_arrays)
            arr = lambda a, dt: None if a is None else _p(a)  # noqa: E731
            src = device_arrays
        else:
            src = {k: getattr(P, k) for k in ("diag", "ax", "ay", "az", "row_ptr", "col", "val")}
        if P.layout == PCG_CSR32:
            m.n, m.nnz = P.n, int(P.row_ptr[-1])
            m.row_ptr, m.col, m.val = arr(src["row_ptr"], np.int32), arr(src["col"], np.int32), arr(src["val"], np.float64)
        else:
            m.nx, m.ny, m.nz = P.nx, P.ny, P.nz
            if src.get("diag") is not None:
                m.diag, m.ax, m.ay = arr(src["diag"], np.float64), arr(src["ax"], np.float64), arr(src["ay"], np.float64)
                if P.layout == PCG_STENCIL7_3D:
                    m.az = arr(src["az"], np.float64)
        self.m = m


@dataclass
class SolveResult:
    x: object
    iters: int
    status: int
    final_true_relres: float
    final_rec_relres: float
    rec: np.ndarray
    true: np.ndarray
    gap: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray


class Solver:
    """One pcg_ctx for one operator."""

    def __init__(self, P, flags: int = 0, device_arrays: Optional[dict] = None):
        self.P = P
        self.n = P.n
        self.mat = Matrix(P, device_arrays)
        self.ctx = pcg_create(self.mat.m, flags | (PCG_DEVICE_PTRS if device_arrays is not None else 0))

    def close(self):
        if getattr(self, "ctx", None):
            pcg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, b, x0=None, method="spcg", sigma=0.0, tol=0.0, maxit=100, true_every=0, device=False,
              x_out=None, raise_on_error=True, precision=PCG_FP64) -> SolveResult:
        """b/x0/x_out: numpy arrays (host) or, with device=True, CUDA tensors."""
        m = METHODS[method] if isinstance(method, str) else method
        k = maxit + 1
        hist = {name: np.full(k, np.nan) for name in ("rec", "true", "gap", "alpha", "beta")}
        res = pcg_result()
        res.rec_hist, res.true_hist, res.gap_hist = _p(hist["rec"]), _p(hist["true"]), _p(hist["gap"])
        res.alpha_hist, res.beta_hist = _p(hist["alpha"]), _p(hist["beta"])
        res.true_every = true_every
        if device:
            if x_out is None:
                import torch
                x_out = torch.empty(self.n, dtype=torch.float64, device=b.device)
            s = pcg_solve_device(self.ctx, b, x0, m, sigma, tol, maxit, precision, x_out, res)
        else:
            b = np.ascontiguousarray(b, dtype=np.float64)
            x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
            if x_out is None:
                x_out = np.empty(self.n)
            s = pcg_solve(self.ctx, b, x0, m, sigma, tol, maxit, precision, x_out, res)
        if s not in (PCG_OK, PCG_ENOTCONV, PCG_EBREAKDOWN) and raise_on_error:
            raise PcgError(s, pcg_last_error(self.ctx))
        it = res.iters
        return SolveResult(x_out, it, s, res.final_true_relres, res.final_rec_relres, hist["rec"][:it + 1],
                           hist["true"][:it + 1], hist["gap"][:it + 1], hist["alpha"][:it], hist["beta"][:it])


class Batch:
    """pcg_batch over a list of problems of one operator family (host arrays)."""

    def __init__(self, problems, flags: int = 0, precision: int = PCG_FP64):
        self.mats = [Matrix(P) for P in problems]
        self.n = [P.n for P in problems]
        arr = (pcg_matrix * len(problems))(*[m.m for m in self.mats])
        self._arr = arr
        out = ctypes.c_void_p()
        s = lib().pcg_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(problems), flags, ctypes.byref(out))
        if s != PCG_OK:
            raise PcgError(s, "pcg_batch_create")
        self.h = out.value
        if precision != PCG_FP64:
            s = lib().pcg_batch_set_precision(self.h, precision)
            if s != PCG_OK:
                raise PcgError(s, "pcg_batch_set_precision")

    def set_precision(self, precision: int) -> int:
        return lib().pcg_batch_set_precision(self.h, precision)

    def set_param(self, param: int, value: float) -> int:
        return lib().pcg_batch_set_param(self.h, param, value)

    def close(self):
        if getattr(self, "h", None):
            lib().pcg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @staticmethod
    def _ptrs(arrays):
        return (ctypes.c_void_p * len(arrays))(*[a.ctypes.data for a in arrays])

    def solve(self, bs, sigma, tol=0.0, maxit=1000, method=PCG_SPCG):
        bs = [np.ascontiguousarray(b, dtype=np.float64) for b in bs]
        xs = [np.empty(n) for n in self.n]
        sg = np.ascontiguousarray(sigma, dtype=np.float64)
        k = len(bs)
        it = np.zeros(k, dtype=np.int32)
        st = np.zeros(k, dtype=np.int32)
        tr = np.zeros(k)
        s = lib().pcg_batch_solve(self.h, ctypes.cast(self._ptrs(bs), ctypes.c_void_p),
                                  ctypes.cast(self._ptrs(xs), ctypes.c_void_p), method, sg.ctypes.data, tol, maxit,
                                  it.ctypes.data, st.ctypes.data, tr.ctypes.data)
        if s not in (PCG_OK, PCG_ENOTCONV):
            raise PcgError(s, "pcg_batch_solve")
        return xs, it, st, tr

    def autotune(self, bs, sigma, probe_iters=50):
        bs = [np.ascontiguousarray(b, dtype=np.float64) for b in bs]
        sg = np.ascontiguousarray(sigma, dtype=np.float64)
        c = ctypes.c_int32()
        ms = np.zeros(5)
        s = lib().pcg_batch_autotune(self.h, ctypes.cast(self._ptrs(bs), ctypes.c_void_p), sg.ctypes.data,
                                     probe_iters, ctypes.byref(c), ms.ctypes.data)
        if s != PCG_OK:
            raise PcgError(s, "pcg_batch_autotune")
        return c.value, ms

    def set_cluster(self, c):
        return lib().pcg_batch_set_cluster(self.h, c)

    def classes(self):
        """(systems per size class, cluster size per class, resident blocks per SM per class)."""
        n = np.zeros(3, dtype=np.int32)
        c = np.zeros(3, dtype=np.int32)
        o = np.zeros(3, dtype=np.int32)
        lib().pcg_batch_classes(self.h, n.ctypes.data, c.ctypes.data, o.ctypes.data)
        return n, c, o

    def set_class_cluster(self, size_class: int, c: int) -> int:
        return lib().pcg_batch_set_class_cluster(self.h, size_class, c)

    def set_class_occupancy(self, size_class: int, blocks_per_sm: int) -> int:
        return lib().pcg_batch_set_class_occupancy(self.h, size_class, blocks_per_sm)

    def last_kernel_ms(self):
        v = ctypes.c_double()
        lib().pcg_batch_last_kernel_ms(self.h, ctypes.byref(v))
        return v.value

    def scalars(self, k: int = PCG_SCALAR_LOG):
        """alpha_i, beta_i (i < k) of every system of the last solve: two (nsys, k) arrays."""
        a = np.empty((len(self.n), k))
        b = np.empty((len(self.n), k))
        s = lib().pcg_batch_scalars(self.h, k, a.ctypes.data, b.ctypes.data)
        if s != PCG_OK:
            raise PcgError(s, "pcg_batch_scalars")
        return a, b


class Server:
    """pcg_server: continuous batching of solve requests (host arrays in and out)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int):
        out = ctypes.c_void_p()
        s = lib().pcg_server_create(hbm_budget_bytes, max_slots, ctypes.byref(out))
        if s != PCG_OK:
            raise PcgError(s, "pcg_server_create")
        self.h = out.value
        self.n = {}

    def close(self):
        if getattr(self, "h", None):
            lib().pcg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, P, b, tol=1e-8, method=PCG_SPCG, sigma=-1.0, maxit=100000, flags=0, precision=PCG_FP64) -> int:
        m = Matrix(P)
        b = np.ascontiguousarray(b, dtype=np.float64)
        t = ctypes.c_uint64()
        s = lib().pcg_submit_ex(self.h, ctypes.byref(m.m), b.ctypes.data, tol, method, sigma, maxit, flags, precision,
                                ctypes.byref(t))
        if s != PCG_OK:
            raise PcgError(s, "pcg_submit")
        self.n[t.value] = P.n
        return t.value

    def poll(self, ticket: int, scalars: bool = False):
        """None while pending, else (status, x, iters, true_relres), and with scalars=True
        also alpha_i, beta_i (i < min(iters, PCG_SCALAR_LOG)) as two arrays."""
        x = np.empty(self.n[ticket])
        res = pcg_result()
        if scalars:
            al = np.full(PCG_SCALAR_LOG, np.nan)
            be = np.full(PCG_SCALAR_LOG, np.nan)
            res.alpha_hist, res.beta_hist = al.ctypes.data, be.ctypes.data
        s = lib().pcg_poll(self.h, ticket, x.ctypes.data, ctypes.byref(res))
        if s == PCG_PENDING:
            return None
        if s not in (PCG_OK, PCG_ENOTCONV, PCG_EBREAKDOWN):
            raise PcgError(s, "pcg_poll")
        del self.n[ticket]
        if scalars:
            m = min(res.iters, PCG_SCALAR_LOG)
            return s, x, res.iters, res.final_true_relres, al[:m], be[:m]
        return s, x, res.iters, res.final_true_relres

    def stats(self):
        w, i, f = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t()
        lib().pcg_server_stats(self.h, ctypes.byref(w), ctypes.byref(i), ctypes.byref(f))
        return w.value, i.value, f.value

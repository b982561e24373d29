"""One system on several GPUs: z-slabs of the 3D 7-point Laplacian, one per rank.

The paper's own setting (Section 1; the MPI runs of Section 5.2): each rank owns whole z
planes of the grid, the SpMV needs one plane of its neighbours on each side, and the dot
products need one global reduction of two scalars per iteration.  The phases of
Algorithm 3 run as kernels of the C ABI (pcg_slab_*, include/pcg.h); this module only
moves data between them:

  * `z_slabs` cuts the grid's planes into contiguous slabs;
  * `CudaSlab` holds one rank's vectors (torch tensors) and calls the slab kernels;
  * `DistComm` exchanges halo planes and reduces the dots with torch.distributed (NCCL
    between GPUs, gloo on CPU ranks);
  * `LocalComm` does the same between slabs held by one process (all on one GPU), so
    the sharded iteration can be checked against the single-system solver and the oracle
    on a single device: the slab kernels never wait on each other, only the host orders
    the copies between them;
  * `solve` runs the iteration on every slab of a communicator.

The order of the phases hides the global reduction behind the SpMV, as in pipelined CG:
the reduction of (gamma_i, omega_i) and the halo exchange of w_i are started, the SpMV
runs on the interior planes, then on the two boundary planes once the halo has arrived,
and only the scalar step waits for the reduction.
"""
from __future__ import annotations

import ctypes
from typing import List, Sequence, Tuple

import numpy as np

from . import pcg as C

PCG_SLAB_X, PCG_SLAB_R, PCG_SLAB_W, PCG_SLAB_N = 0, 1, 2, 3
ALL, INTERIOR, BOUNDARY = 0, 1, 2


def z_slabs(nz: int, world: int) -> List[Tuple[int, int]]:
    """Planes [k0, k1) of each rank: contiguous, sizes differing by at most one plane."""
    if world < 1 or nz < world:
        raise ValueError("need at least one plane per rank")
    base, extra = divmod(nz, world)
    out, k = [], 0
    for r in range(world):
        m = base + (1 if r < extra else 0)
        out.append((k, k + m))
        k += m
    return out


class pcg_slab_vectors(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("x", "r", "w", "z", "s", "p", "n", "b", "halo_below", "halo_above")]


def _declare(L):
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    if getattr(L, "_slab_declared", False):
        return L
    L.pcg_slab_create.argtypes = [i64, i64, i64, i32, i32, ctypes.POINTER(pcg_slab_vectors), i32,
                                  ctypes.POINTER(vp)]
    L.pcg_slab_set_stream.argtypes = [vp, vp]
    L.pcg_slab_start.argtypes = [vp, f64, f64, vp]
    L.pcg_slab_set_bnorm.argtypes = [vp, vp]
    L.pcg_slab_spmv.argtypes = [vp, i32, i32, i32]
    L.pcg_slab_w0.argtypes = [vp, vp]
    L.pcg_slab_scalars.argtypes = [vp, vp, i32]
    L.pcg_slab_update.argtypes = [vp, vp]
    L.pcg_slab_true_residual.argtypes = [vp, vp]
    L.pcg_slab_state.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(f64)]
    L.pcg_slab_history.argtypes = [vp, i32, vp, vp, vp]
    L.pcg_slab_last_error.argtypes = [vp]
    L.pcg_slab_last_error.restype = ctypes.c_char_p
    L.pcg_slab_destroy.argtypes = [vp]
    L.pcg_slab_destroy.restype = None
    for f in ("pcg_slab_create", "pcg_slab_set_stream", "pcg_slab_start", "pcg_slab_set_bnorm", "pcg_slab_spmv",
              "pcg_slab_w0", "pcg_slab_scalars", "pcg_slab_update", "pcg_slab_true_residual", "pcg_slab_state",
              "pcg_slab_history"):
        getattr(L, f).restype = ctypes.c_int
    L._slab_declared = True
    return L


class CudaSlab:
    """One rank's slab on the current CUDA device: planes [k0, k1) of an nx x ny x nz
    grid, its vectors as torch tensors, the phases as pcg_slab_* kernels."""

    VECS = ("x", "r", "w", "z", "s", "p", "n")

    def __init__(self, nx: int, ny: int, k0: int, k1: int, nz: int, b_local, maxit: int, stream=None):
        import torch
        self.nx, self.ny, self.k0, self.k1, self.nz = nx, ny, k0, k1, nz
        self.nzl = k1 - k0
        self.plane_size = nx * ny
        n = self.plane_size * self.nzl
        dev = torch.device("cuda", torch.cuda.current_device())
        self.b = torch.as_tensor(b_local, dtype=torch.float64).to(dev).contiguous()
        assert self.b.numel() == n
        self.v = {k: torch.empty(n, dtype=torch.float64, device=dev) for k in self.VECS}
        self.halo_lo = torch.zeros(self.plane_size, dtype=torch.float64, device=dev)
        self.halo_hi = torch.zeros(self.plane_size, dtype=torch.float64, device=dev)
        self.dots = torch.zeros(2, dtype=torch.float64, device=dev)
        self.has_lo, self.has_hi = k0 > 0, k1 < nz
        vv = pcg_slab_vectors(*[self.v[k].data_ptr() for k in self.VECS], self.b.data_ptr(),
                              self.halo_lo.data_ptr(), self.halo_hi.data_ptr())
        self.L = _declare(C.lib())
        h = ctypes.c_void_p()
        s = self.L.pcg_slab_create(nx, ny, self.nzl, int(self.has_lo), int(self.has_hi), ctypes.byref(vv), maxit,
                                   ctypes.byref(h))
        if s != C.PCG_OK:
            raise C.PcgError(s, "pcg_slab_create")
        self.h = h.value
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.L.pcg_slab_set_stream(self.h, self.stream.cuda_stream)

    def _ok(self, s, what):
        if s != C.PCG_OK:
            raise C.PcgError(s, f"{what}: {self.L.pcg_slab_last_error(self.h).decode()}")

    def plane(self, name: str, k: int):
        """Plane k (local index) of vector `name`, a view."""
        return self.v[name][k * self.plane_size:(k + 1) * self.plane_size]

    def start(self, sigma: float, tol: float):
        self._ok(self.L.pcg_slab_start(self.h, sigma, tol, self.dots.data_ptr()), "start")

    def set_bnorm(self):
        self._ok(self.L.pcg_slab_set_bnorm(self.h, self.dots.data_ptr()), "set_bnorm")

    def spmv(self, src: int, dst: int, planes: int):
        self._ok(self.L.pcg_slab_spmv(self.h, src, dst, planes), "spmv")

    def w0(self):
        self._ok(self.L.pcg_slab_w0(self.h, self.dots.data_ptr()), "w0")

    def scalars(self, first: bool):
        self._ok(self.L.pcg_slab_scalars(self.h, self.dots.data_ptr(), int(first)), "scalars")

    def update(self):
        self._ok(self.L.pcg_slab_update(self.h, self.dots.data_ptr()), "update")

    def true_residual(self):
        self._ok(self.L.pcg_slab_true_residual(self.h, self.dots.data_ptr()), "true_residual")

    def state(self):
        it, st, bn = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        self._ok(self.L.pcg_slab_state(self.h, ctypes.byref(it), ctypes.byref(st), ctypes.byref(bn)), "state")
        return it.value, st.value, bn.value

    def history(self, k: int):
        a, b, r = np.full(k, np.nan), np.full(k, np.nan), np.full(k, np.nan)
        self._ok(self.L.pcg_slab_history(self.h, k, a.ctypes.data, b.ctypes.data, r.ctypes.data), "history")
        return a, b, r

    def x_host(self) -> np.ndarray:
        return self.v["x"].cpu().numpy()

    def close(self):
        if getattr(self, "h", None):
            self.L.pcg_slab_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


class _Done:
    def wait(self):
        return None


class DistComm:
    """Halo exchange and dot reduction between ranks of torch.distributed (one slab per
    process; NCCL between GPUs, gloo on CPU ranks)."""

    def __init__(self, rank: int, world: int, group=None):
        self.rank, self.world, self.group = rank, world, group

    def exchange(self, slab, name: str):
        """Starts moving the boundary planes of vector `name` into the neighbours' halos;
        returns an object whose wait() completes the exchange."""
        import torch.distributed as dist
        works = []
        if slab.has_lo:
            works.append(dist.irecv(slab.halo_lo, self.rank - 1, group=self.group))
            works.append(dist.isend(slab.plane(name, 0).contiguous(), self.rank - 1, group=self.group))
        if slab.has_hi:
            works.append(dist.irecv(slab.halo_hi, self.rank + 1, group=self.group))
            works.append(dist.isend(slab.plane(name, slab.nzl - 1).contiguous(), self.rank + 1, group=self.group))

        class _W:
            def wait(self_inner):
                for w in works:
                    w.wait()
        return _W()

    def allreduce(self, slab):
        """Starts summing every rank's slab.dots into slab.dots."""
        import torch.distributed as dist
        return dist.all_reduce(slab.dots, group=self.group, async_op=True)


class LocalComm:
    """The same between slabs held by this process: copies between their tensors, and the
    dots summed in rank order.  Phases are stepped for every slab in turn."""

    def __init__(self, slabs: Sequence):
        self.slabs = list(slabs)

    def exchange_all(self, name: str):
        for r, s in enumerate(self.slabs):
            if s.has_lo:
                s.halo_lo.copy_(self.slabs[r - 1].plane(name, self.slabs[r - 1].nzl - 1))
            if s.has_hi:
                s.halo_hi.copy_(self.slabs[r + 1].plane(name, 0))

    def allreduce_all(self):
        tot = self.slabs[0].dots.clone()
        for s in self.slabs[1:]:
            tot = tot + s.dots
        for s in self.slabs:
            s.dots.copy_(tot)


def solve_rank(slab, comm: DistComm, sigma: float, tol: float, maxit: int, check_every: int = 50) -> dict:
    """Algorithm 3 on this rank's slab, the other ranks running the same call."""
    slab.start(sigma, tol)
    comm.allreduce(slab).wait()
    slab.set_bnorm()
    comm.exchange(slab, "r").wait()
    slab.spmv(PCG_SLAB_R, PCG_SLAB_W, ALL)
    slab.w0()
    for i in range(maxit + 1):
        red = comm.allreduce(slab)              # gamma_i, omega_i: hidden behind the SpMV
        ex = comm.exchange(slab, "w")
        slab.spmv(PCG_SLAB_W, PCG_SLAB_N, INTERIOR)
        ex.wait()
        slab.spmv(PCG_SLAB_W, PCG_SLAB_N, BOUNDARY)
        red.wait()
        slab.scalars(i == 0)
        slab.update()
        if check_every and (i + 1) % check_every == 0 and slab.state()[1] != C.PCG_PENDING:
            break
    it, status, bnorm = slab.state()
    comm.exchange(slab, "x").wait()
    slab.spmv(PCG_SLAB_X, PCG_SLAB_N, ALL)
    slab.true_residual()
    comm.allreduce(slab).wait()
    d = slab.dots.cpu().numpy()
    return {"iters": it, "status": status, "bnorm": bnorm, "true_relres": float(np.sqrt(d[0])) / bnorm,
            "gap_rel": float(np.sqrt(d[1])) / bnorm}


def solve_local(slabs: Sequence, sigma: float, tol: float, maxit: int, check_every: int = 50) -> dict:
    """The same iteration for every slab held by this process (LocalComm), phase by phase."""
    comm = LocalComm(slabs)
    for s in slabs:
        s.start(sigma, tol)
    comm.allreduce_all()
    for s in slabs:
        s.set_bnorm()
    comm.exchange_all("r")
    for s in slabs:
        s.spmv(PCG_SLAB_R, PCG_SLAB_W, ALL)
        s.w0()
    for i in range(maxit + 1):
        comm.allreduce_all()
        for s in slabs:
            s.spmv(PCG_SLAB_W, PCG_SLAB_N, INTERIOR)
        comm.exchange_all("w")
        for s in slabs:
            s.spmv(PCG_SLAB_W, PCG_SLAB_N, BOUNDARY)
            s.scalars(i == 0)
            s.update()
        if check_every and (i + 1) % check_every == 0 and slabs[0].state()[1] != C.PCG_PENDING:
            break
    it, status, bnorm = slabs[0].state()
    comm.exchange_all("x")
    for s in slabs:
        s.spmv(PCG_SLAB_X, PCG_SLAB_N, ALL)
        s.true_residual()
    comm.allreduce_all()
    d = slabs[0].dots.cpu().numpy()
    return {"iters": it, "status": status, "bnorm": bnorm, "true_relres": float(np.sqrt(d[0])) / bnorm,
            "gap_rel": float(np.sqrt(d[1])) / bnorm}

"""One system on several ranks (z-slabs, halo planes, one 2-scalar reduction per
iteration): the host logic of paper_1706_05988_gb300/sharded.py on gloo ranks on the CPU.

Each rank runs sharded.solve_rank -- the same driver and the same torch.distributed
exchange the GPU ranks use -- with a CPU stand-in for its slab's kernels (CpuSlab below:
the phases written out in float64 numpy, no shared code with the oracle or the CUDA
kernels).  The concatenated iterate and the scalars must be the oracle's Algorithm 3 on the
whole grid."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class CpuSlab:
    """The slab phases of pcg_slab_* written out plainly (test-side stand-in for the
    kernels; float64, torch CPU tensors so that torch.distributed can move them)."""

    def __init__(self, nx, ny, k0, k1, nz, b_local, maxit):
        import torch
        self.nx, self.ny, self.k0, self.k1, self.nz, self.nzl = nx, ny, k0, k1, nz, k1 - k0
        self.plane_size = nx * ny
        self.maxit = maxit
        n = self.plane_size * self.nzl
        self.b = torch.as_tensor(np.asarray(b_local, dtype=np.float64)).clone()
        self.v = {k: torch.zeros(n, dtype=torch.float64) for k in ("x", "r", "w", "z", "s", "p", "n")}
        self.halo_lo = torch.zeros(self.plane_size, dtype=torch.float64)
        self.halo_hi = torch.zeros(self.plane_size, dtype=torch.float64)
        self.dots = torch.zeros(2, dtype=torch.float64)
        self.has_lo, self.has_hi = k0 > 0, k1 < nz
        self.alpha, self.beta, self.rec = [], [], []
        self.status, self.iter = 7, 0

    def plane(self, name, k):
        return self.v[name][k * self.plane_size:(k + 1) * self.plane_size]

    def _a(self, src, kb, ke):
        """(A src) on planes [kb, ke): 6 w_c - neighbours, halos at the slab's ends."""
        u = src.numpy().reshape(self.nzl, self.ny, self.nx)
        lo = self.halo_lo.numpy().reshape(self.ny, self.nx) if self.has_lo else np.zeros((self.ny, self.nx))
        hi = self.halo_hi.numpy().reshape(self.ny, self.nx) if self.has_hi else np.zeros((self.ny, self.nx))
        ext = np.concatenate([lo[None], u, hi[None]], axis=0)
        y = 6.0 * ext[1:-1].copy()
        y -= ext[:-2] + ext[2:]
        y[:, 1:, :] -= u[:, :-1, :]
        y[:, :-1, :] -= u[:, 1:, :]
        y[:, :, 1:] -= u[:, :, :-1]
        y[:, :, :-1] -= u[:, :, 1:]
        return y.reshape(-1)[kb * self.plane_size:ke * self.plane_size]

    def start(self, sigma, tol):
        self.sigma, self.tol = sigma, tol
        self.v["r"][:] = self.b
        for k in ("x", "z", "s", "p"):
            self.v[k][:] = 0.0
        self.dots[:] = 0.0
        self.dots[0] = float(np.dot(self.b.numpy(), self.b.numpy()))
        self.status, self.iter = 7, 0
        self.alpha, self.beta, self.rec = [], [], []

    def set_bnorm(self):
        self.bnorm = float(np.sqrt(float(self.dots[0])))

    def spmv(self, src, dst, planes):
        import torch
        names = {0: "x", 1: "r", 2: "w", 3: "n"}
        if planes == 0:
            segs = [(0, self.nzl)]
        elif planes == 1:
            segs = [(1, self.nzl - 1)]
        else:
            segs = [(0, 1), (self.nzl - 1, self.nzl)]
        for kb, ke in segs:
            if kb < ke:
                y = torch.as_tensor(self._a(self.v[names[src]], kb, ke))
                self.v[names[dst]][kb * self.plane_size:ke * self.plane_size] = y

    def w0(self):
        r, w = self.v["r"].numpy(), self.v["w"].numpy()
        w -= self.sigma * r
        self.dots[0], self.dots[1] = float(np.dot(r, r)), float(np.dot(w, r))

    def scalars(self, first):
        if self.status != 7:
            return
        g, om = float(self.dots[0]), float(self.dots[1])
        i = 0 if first else self.iter + 1
        d = om + self.sigma * g
        self.rec.append(np.sqrt(g))
        self.iter = i
        if self.tol > 0 and np.sqrt(g) <= self.tol * self.bnorm:
            self.status = 0
        elif i >= self.maxit:
            self.status = 5
        elif g == 0.0:
            self.status = 0
        elif first:
            self.alpha.append(g / d)
            self.beta.append(0.0)
        else:
            bt = g / self.gprev
            self.alpha.append(1.0 / (d / g - bt / self.alpha[-1]))
            self.beta.append(bt)
        self.gprev = g

    def update(self):
        if self.status != 7:
            return
        a, bt, sg = self.alpha[-1], self.beta[-1], self.sigma
        v = {k: t.numpy() for k, t in self.v.items()}
        v["z"][:] = v["n"] + bt * v["z"]
        v["s"][:] = v["w"] + bt * v["s"]
        v["p"][:] = v["r"] + bt * v["p"]
        v["x"][:] = v["x"] + a * v["p"]
        v["r"][:] = v["r"] - (a * v["s"] + a * sg * v["p"])
        v["w"][:] = v["w"] - a * v["z"]
        self.dots[0], self.dots[1] = float(np.dot(v["r"], v["r"])), float(np.dot(v["w"], v["r"]))

    def true_residual(self):
        t = self.b.numpy() - self.v["n"].numpy()
        f = t - self.v["r"].numpy()
        self.dots[0], self.dots[1] = float(np.dot(t, t)), float(np.dot(f, f))

    def state(self):
        return self.iter, self.status, self.bnorm

    def history(self, k):
        out = [np.full(k, np.nan) for _ in range(3)]
        for arr, src in zip(out, (self.alpha, self.beta, self.rec)):
            m = min(k, len(src))
            arr[:m] = src[:m]
        return tuple(out)


GRID = (10, 9, 13)       # nx, ny, nz of the global grid
MAXIT = 20
SIGMA = 6.0


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    from paper_1706_05988_gb300 import sharded as SH
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nx, ny, nz = GRID
    P = S.laplacian_3d(nx, ny, nz)
    b = S.normal(21, P.n)
    k0, k1 = SH.z_slabs(nz, world)[rank]
    slab = CpuSlab(nx, ny, k0, k1, nz, b[k0 * nx * ny:k1 * nx * ny], MAXIT)
    res = SH.solve_rank(slab, SH.DistComm(rank, world), SIGMA, 0.0, MAXIT, check_every=0)
    a, bt, _ = slab.history(MAXIT)
    out[rank] = (k0, k1, slab.v["x"].numpy().copy(), a, bt, res)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_gloo_ranks_vs_oracle(world):
    import torch.multiprocessing as mp
    import oracle
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    nx, ny, nz = GRID
    P = S.laplacian_3d(nx, ny, nz)
    b = S.normal(21, P.n)
    o = oracle.pcg_sh(P, b, sigma=SIGMA, maxit=MAXIT, log_every=MAXIT)
    x = np.concatenate([res[r][2] for r in range(world)])
    assert [(res[r][0], res[r][1]) for r in range(world)] == SH_slabs(nz, world)
    for r in range(world):
        a, bt, rr = res[r][3], res[r][4], res[r][5]
        assert rr["iters"] == MAXIT and rr["status"] == 5            # PCG_ENOTCONV: maxit reached
        assert np.max(np.abs(a - o.alpha) / np.abs(o.alpha)) <= 1e-10
        assert np.max(np.abs(bt[1:] - o.beta[1:]) / np.abs(o.beta[1:])) <= 1e-10
        bn = np.linalg.norm(b)
        assert abs(rr["true_relres"] - o.true[-1] / bn) <= 1e-9 * o.true[-1] / bn
    assert np.linalg.norm(x - o.x) <= 1e-11 * np.linalg.norm(o.x)


def SH_slabs(nz, world):
    from paper_1706_05988_gb300 import sharded as SH
    return SH.z_slabs(nz, world)


def test_z_slabs_partition():
    from paper_1706_05988_gb300 import sharded as SH
    for nz in (1, 5, 13, 256):
        for world in range(1, min(nz, 9) + 1):
            sl = SH.z_slabs(nz, world)
            assert sl[0][0] == 0 and sl[-1][1] == nz
            assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
            sizes = [k1 - k0 for k0, k1 in sl]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        SH.z_slabs(3, 4)


def test_cpu_slab_stand_in_single_rank_vs_oracle():
    """The stand-in itself on one rank (no halo): the oracle's scalars, so that the ranked
    tests check the exchange and the reduction, not the stand-in."""
    import oracle
    from paper_1706_05988_gb300 import sharded as SH

    class NoComm:
        def exchange(self, slab, name):
            return SH._Done()

        def allreduce(self, slab):
            return SH._Done()

    nx, ny, nz = GRID
    P = S.laplacian_3d(nx, ny, nz)
    b = S.normal(21, P.n)
    slab = CpuSlab(nx, ny, 0, nz, nz, b, MAXIT)
    SH.solve_rank(slab, NoComm(), SIGMA, 0.0, MAXIT, check_every=0)
    o = oracle.pcg_sh(P, b, sigma=SIGMA, maxit=MAXIT, log_every=0)
    a, bt, _ = slab.history(MAXIT)
    assert np.max(np.abs(a - o.alpha) / np.abs(o.alpha)) <= 1e-10
    assert np.linalg.norm(slab.v["x"].numpy() - o.x) <= 1e-11 * np.linalg.norm(o.x)

"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds problem *data* only: random numbers, grids, coefficient
fields and the sparse pattern of the model operators.  It contains none of the
solver's arithmetic (no Krylov recurrence, no dot product, no scalar update).

Random numbers come from one counter-based generator, SplitMix64
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): value k of stream `seed` is mix64(seed + (k + 1) * 0x9E3779B97F4A7C15).

Model problems (the paper's Section 5 uses the unscaled 2D Laplacian
`lapl200` and PETSc's 2D Poisson example; the larger shapes follow the same
discretisation):

* constant-coefficient Dirichlet Laplacians on nx x ny (5-point, diagonal 4,
  off-diagonals -1) and nx x ny x nz grids (7-point, diagonal 6), no 1/h^2
  scaling, x index fastest in memory;
* variable-coefficient cell-centred finite-volume diffusion: face
  transmissibility 2*k_a*k_b/(k_a+k_b), Dirichlet boundary face 2*k_cell,
  diagonal = sum of the cell's face transmissibilities;
* the same operators assembled as CSR with int32 indices.

Right-hand sides b = A x* are formed only for the constant-coefficient
Laplacians and only from x* on the dyadic grid 2^-30 Z inside [-1, 1]: every
product and partial sum of 6 x_c - sum(neighbours) is then an exact binary64
number, so b is the same bit pattern whatever order anyone sums in.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Layout codes, identical to the C-ABI's pcg_layout values.
STENCIL5_2D = 0
STENCIL7_3D = 1
CSR32 = 2

DYADIC_BITS = 30


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Values offset .. offset+count-1 of the SplitMix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """U[0,1) from the top 53 bits of each SplitMix64 value."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """U[-1,1) with 53-bit resolution."""
    return 2.0 * uniform01(seed, count, offset) - 1.0


def dyadic_uniform_pm1(seed: int, count: int, bits: int = DYADIC_BITS, offset: int = 0) -> np.ndarray:
    """U[-1,1) rounded down to the grid 2^-bits (exactly representable, |v| <= 1); values
    offset .. offset+count-1 of the stream."""
    u = splitmix64(seed, count, offset) >> np.uint64(64 - (bits + 1))   # integer in [0, 2^(bits+1))
    return (u.astype(np.int64) - (1 << bits)).astype(np.float64) * (2.0 ** -bits)


def normal(seed: int, count: int) -> np.ndarray:
    """N(0,1) by the Box-Muller transform of consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]                     # (0, 1]: log is finite
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = rad * np.cos(2.0 * np.pi * u2)
    out[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return out[:count]


@dataclass
class Problem:
    """A model SPD operator.  Stencil problems carry dims; variable-coefficient
    problems carry per-cell face coefficients (all float64, length n):

    diag[c]           diagonal entry of row c
    ax[c], ay[c], az[c]  transmissibility of the face between c and its lower
                      x / y / z neighbour (0 on the domain boundary, whose
                      Dirichlet contribution is already inside diag)
    Constant-coefficient Laplacians have coef arrays = None.
    CSR problems carry row_ptr/col/val (int32, int32, float64)."""

    layout: int
    nx: int = 0
    ny: int = 1
    nz: int = 1
    diag: Optional[np.ndarray] = None
    ax: Optional[np.ndarray] = None
    ay: Optional[np.ndarray] = None
    az: Optional[np.ndarray] = None
    row_ptr: Optional[np.ndarray] = None
    col: Optional[np.ndarray] = None
    val: Optional[np.ndarray] = None
    n_csr: int = 0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        if self.layout == CSR32:
            return self.n_csr
        return self.nx * self.ny * self.nz

    @property
    def is_3d(self) -> bool:
        return self.layout == STENCIL7_3D

    @property
    def constant(self) -> bool:
        return self.diag is None

    @property
    def nnz(self) -> int:
        if self.layout == CSR32:
            return int(self.row_ptr[-1])
        return _stencil_nnz(self.nx, self.ny, self.nz, self.is_3d)


def _stencil_nnz(nx, ny, nz, is3d):
    nnz = nx * ny * nz + 2 * ((nx - 1) * ny * nz + nx * (ny - 1) * nz)
    if is3d:
        nnz += 2 * nx * ny * (nz - 1)
    return nnz


def laplacian_2d(nx: int, ny: Optional[int] = None) -> Problem:
    """Unscaled 5-point Dirichlet Laplacian: 4 on the diagonal, -1 to each grid neighbour."""
    return Problem(STENCIL5_2D, nx, ny if ny is not None else nx, 1, name=f"lapl2d_{nx}")


def laplacian_3d(nx: int, ny: Optional[int] = None, nz: Optional[int] = None) -> Problem:
    """Unscaled 7-point Dirichlet Laplacian: 6 on the diagonal, -1 to each grid neighbour."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return Problem(STENCIL7_3D, nx, ny, nz, name=f"lapl3d_{nx}")


def _fv_faces(kappa: np.ndarray):
    """Face transmissibilities of a cell-centred FV diffusion operator on a
    (nz, ny, nx) kappa field: harmonic mean between cells, 2*kappa at a Dirichlet face."""
    def hmean(a, b):
        return 2.0 * a * b / (a + b)

    shape = kappa.shape
    faces = []
    diag = np.zeros(shape)
    for axis in range(kappa.ndim):
        lower = np.zeros(shape)                 # face between c and c - e_axis
        sl_hi = [slice(None)] * kappa.ndim
        sl_lo = [slice(None)] * kappa.ndim
        sl_hi[axis] = slice(1, None)
        sl_lo[axis] = slice(0, -1)
        t = hmean(kappa[tuple(sl_lo)], kappa[tuple(sl_hi)])
        lower[tuple(sl_hi)] = t
        faces.append(lower)
        # diagonal: interior faces on both sides, plus 2*kappa at the two boundary faces
        diag[tuple(sl_hi)] += t
        diag[tuple(sl_lo)] += t
        first = [slice(None)] * kappa.ndim
        last = [slice(None)] * kappa.ndim
        first[axis] = 0
        last[axis] = -1
        diag[tuple(first)] += 2.0 * kappa[tuple(first)]
        diag[tuple(last)] += 2.0 * kappa[tuple(last)]
    return diag, faces


def varcoef_3d(n: int, block: int = 8, lo_exp: float = -3.0, hi_exp: float = 3.0, seed: int = 0) -> Problem:
    """7-point FV diffusion on n^3 cells, kappa constant on block^3 blocks, 10^U[lo,hi] per block."""
    nb = (n + block - 1) // block
    e = lo_exp + (hi_exp - lo_exp) * uniform01(seed, nb ** 3).reshape(nb, nb, nb)
    kb = 10.0 ** e
    kappa = np.repeat(np.repeat(np.repeat(kb, block, 0), block, 1), block, 2)[:n, :n, :n]
    diag, (fx, fy, fz) = _fv_faces(np.ascontiguousarray(kappa))
    # faces list order follows numpy axes (z, y, x)
    return Problem(STENCIL7_3D, n, n, n, diag=diag.ravel(), ax=fz.ravel(), ay=fy.ravel(), az=fx.ravel(),
                   name=f"varcoef3d_{n}", meta={"kappa": kappa})


def varcoef_2d(nx: int, ny: Optional[int] = None, lo_exp: float = -2.0, hi_exp: float = 2.0, seed: int = 0) -> Problem:
    """5-point FV diffusion on nx x ny cells, kappa = 10^U[lo,hi] per cell."""
    ny = nx if ny is None else ny
    e = lo_exp + (hi_exp - lo_exp) * uniform01(seed, nx * ny).reshape(ny, nx)
    kappa = 10.0 ** e
    diag, (fy, fx) = _fv_faces(kappa)
    return Problem(STENCIL5_2D, nx, ny, 1, diag=diag.ravel(), ax=fx.ravel(), ay=fy.ravel(),
                   az=np.zeros(nx * ny), name=f"varcoef2d_{nx}x{ny}", meta={"kappa": kappa})


def to_csr(p: Problem) -> Problem:
    """Assemble a stencil problem as CSR (int32 indices, columns ascending per row)."""
    if p.layout == CSR32:
        return p
    nx, ny, nz = p.nx, p.ny, p.nz
    n = nx * ny * nz
    c = np.arange(n, dtype=np.int64)
    i = c % nx
    j = (c // nx) % ny
    k = c // (nx * ny)
    if p.constant:
        centre = 6.0 if p.is_3d else 4.0
        diag = np.full(n, centre)
        one = np.ones(n)
        ax = ay = az = one
    else:
        diag, ax, ay, az = p.diag, p.ax, p.ay, p.az
    nxny = nx * ny
    # candidate entries of every row, in ascending column order
    cand, vals, ok = [], [], []
    if p.is_3d:
        cand.append(c - nxny); ok.append(k > 0); vals.append(-az)
    cand.append(c - nx); ok.append(j > 0); vals.append(-ay)
    cand.append(c - 1); ok.append(i > 0); vals.append(-ax)
    cand.append(c); ok.append(np.ones(n, dtype=bool)); vals.append(diag)
    up = lambda a, off: np.concatenate([a[off:], np.zeros(off)])  # noqa: E731  coefficient of the upper face
    cand.append(c + 1); ok.append(i < nx - 1); vals.append(-up(ax, 1))
    cand.append(c + nx); ok.append(j < ny - 1); vals.append(-up(ay, nx))
    if p.is_3d:
        cand.append(c + nxny); ok.append(k < nz - 1); vals.append(-up(az, nxny))
    mask = np.stack(ok, axis=1)
    col = np.stack(cand, axis=1)[mask]
    val = np.stack(vals, axis=1)[mask]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(mask.sum(axis=1), out=row_ptr[1:])
    assert row_ptr[-1] < 2 ** 31
    return Problem(CSR32, row_ptr=row_ptr.astype(np.int32), col=col.astype(np.int32),
                   val=np.ascontiguousarray(val, dtype=np.float64), n_csr=n, name=p.name + "_csr",
                   meta={"from": p.name, "nx": nx, "ny": ny, "nz": nz})


def _sdd_draws(n: int, seed: int, nnz_lo: int, nnz_hi: int):
    """The random draws of random_sdd_csr: upper partners and their values."""
    d = nnz_lo + (splitmix64(seed, n) % np.uint64(nnz_hi - nnz_lo + 1)).astype(np.int64)
    k = (d - 1) // 2
    rows = np.repeat(np.arange(n, dtype=np.int64), k)
    cols = (splitmix64(seed + 1, rows.size) % np.uint64(max(n - 1, 1))).astype(np.int64)
    cols = cols + (cols >= rows)                     # never the diagonal
    vals = -uniform01(seed + 2, rows.size)
    return rows, cols, vals


def _i64(u: int) -> int:
    """The int64 with the bits of uint64 u."""
    return int(np.array(u, dtype=np.uint64).view(np.int64))


def _splitmix64_t(seed: int, count: int, dev):
    """splitmix64(seed, count) as an int64 torch tensor holding the same 64 bits (wrapping
    int64 arithmetic; >> made logical with a mask)."""
    import torch

    def lsr(z, sh):
        return (z >> sh) & ((1 << (64 - sh)) - 1)

    z = torch.arange(1, count + 1, dtype=torch.int64, device=dev) * _i64(int(GOLDEN)) + _i64(seed)
    z = (z ^ lsr(z, 30)) * _i64(int(_M1))
    z = (z ^ lsr(z, 27)) * _i64(int(_M2))
    return z ^ lsr(z, 31)


def _umod_t(z, m: int):
    """(uint64 bits of z) mod m for 0 < m < 2^31, in int64 arithmetic."""
    hi = (z >> 32) & 0xFFFFFFFF
    lo = z & 0xFFFFFFFF
    return ((hi % m) * ((1 << 32) % m) + lo) % m


def _seq_segment_sum(v, start, length, maxlen: int):
    """Sum of each segment v[start : start + length], added left to right (the order of
    numpy's reduceat), with elementwise passes only: the same bits on any device."""
    import torch
    acc = v[start].clone()
    last = v.numel() - 1
    for j in range(1, maxlen):
        idx = torch.clamp(start + j, max=last)
        acc = acc + torch.where(length > j, v[idx], torch.zeros_like(acc))
    return acc


def random_sdd_csr(n: int, seed: int = 0, nnz_lo: int = 7, nnz_hi: int = 27, margin: float = 1e-2) -> Problem:
    """Random symmetric strictly diagonally dominant CSR matrix (SPD).

    Each row draws a target count d ~ U{nnz_lo..nnz_hi} of entries; (d - 1) // 2 partner
    columns are drawn uniformly among the other rows and the pattern is mirrored, so rows
    hold about nnz_lo..nnz_hi entries.  Off-diagonals ~ U[-1, 0] (a pair drawn twice is
    summed); the diagonal is (1 + margin) * sum |off-diagonals| of its row (strict
    dominance makes A SPD).  Columns are sorted within each row.

    Assembly (torch, on a GPU when one is present): the draws are grouped by unordered pair
    with a stable sort and a pair drawn more than once is summed in draw order (so (i, j) and
    (j, i) hold the same bits); the mirrored entries and one diagonal slot per row are then
    ordered by their (row, column) keys, and each row's absolute sum is added left to right.
    Every sum is an explicit left-to-right pass, so the result has the same bits on any
    device and equals random_sdd_csr_numpy's (tested)."""
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    d = nnz_lo + _umod_t(_splitmix64_t(seed, n, dev), nnz_hi - nnz_lo + 1)
    k = (d - 1) // 2
    rows = torch.repeat_interleave(torch.arange(n, dtype=torch.int64, device=dev), k)
    m = rows.numel()
    cols = _umod_t(_splitmix64_t(seed + 1, m, dev), max(n - 1, 1))
    cols = cols + (cols >= rows).to(torch.int64)
    vals = -(((_splitmix64_t(seed + 2, m, dev) >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53))
    # one value per unordered pair {i, j}: pairs drawn more than once are summed first, in
    # draw order, so that (i, j) and (j, i) hold the same bits
    lo = torch.minimum(rows, cols)
    hi = torch.maximum(rows, cols)
    pkey, perm = torch.sort(lo * n + hi, stable=True)
    pval = vals[perm]
    first = torch.ones_like(pkey, dtype=torch.bool)
    first[1:] = pkey[1:] != pkey[:-1]
    pstart = torch.nonzero(first).flatten()
    plen = torch.diff(pstart, append=torch.tensor([pkey.numel()], device=dev))
    pval = _seq_segment_sum(pval, pstart, plen, int(plen.max()) if plen.numel() else 1)
    pkey = pkey[pstart]
    lo = pkey // n
    hi = pkey - lo * n
    # mirror, add one diagonal slot per row, and order by (row, column)
    diag_idx = torch.arange(n, dtype=torch.int64, device=dev)
    key = torch.cat([lo * n + hi, hi * n + lo, diag_idx * (n + 1)])
    val = torch.cat([pval, pval, torch.zeros(n, dtype=torch.float64, device=dev)])
    key, perm = torch.sort(key)            # keys are unique now
    val = val[perm]
    row = key // n
    col = key - row * n
    counts = torch.bincount(row, minlength=n)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    row_ptr[1:] = torch.cumsum(counts, 0)
    offsum = _seq_segment_sum(val.abs(), row_ptr[:-1], counts, int(counts.max()))   # diagonal slot is 0
    diag = (1.0 + margin) * offsum
    diag[diag == 0] = 1.0
    on_diag = col == row
    val[on_diag] = diag[row[on_diag]]
    assert int(row_ptr[-1]) < 2 ** 31
    return Problem(CSR32, row_ptr=row_ptr.to(torch.int32).cpu().numpy(), col=col.to(torch.int32).cpu().numpy(),
                   val=np.ascontiguousarray(val.cpu().numpy(), dtype=np.float64), n_csr=n, name=f"sdd_{n}")


def _seq_segment_sum_np(v, start, length):
    """_seq_segment_sum in numpy: each segment added left to right."""
    acc = v[start].copy()
    for j in range(1, int(length.max())):
        idx = np.minimum(start + j, v.size - 1)
        acc = acc + np.where(length > j, v[idx], 0.0)
    return acc


def random_sdd_csr_numpy(n: int, seed: int = 0, nnz_lo: int = 7, nnz_hi: int = 27, margin: float = 1e-2) -> Problem:
    """random_sdd_csr in plain numpy (single-threaded; the reference for its bits)."""
    rows, cols, vals = _sdd_draws(n, seed, nnz_lo, nnz_hi)
    lo = np.minimum(rows, cols)
    hi = np.maximum(rows, cols)
    perm = np.argsort(lo * n + hi, kind="stable")
    pkey = (lo * n + hi)[perm]
    pval = vals[perm]
    pstart = np.flatnonzero(np.r_[True, pkey[1:] != pkey[:-1]])
    pval = _seq_segment_sum_np(pval, pstart, np.diff(np.r_[pstart, pkey.size]))
    pkey = pkey[pstart]
    lo = pkey // n
    hi = pkey - lo * n
    diag_idx = np.arange(n, dtype=np.int64)
    key = np.concatenate([lo * n + hi, hi * n + lo, diag_idx * (n + 1)])
    val = np.concatenate([pval, pval, np.zeros(n)])
    perm = np.argsort(key, kind="stable")
    key = key[perm]
    val = val[perm]
    row = key // n
    col = key - row * n
    counts = np.bincount(row, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    offsum = _seq_segment_sum_np(np.abs(val), row_ptr[:-1], counts)
    diag = (1.0 + margin) * offsum
    diag[diag == 0] = 1.0
    on_diag = col == row
    val[on_diag] = diag[row[on_diag]]
    return Problem(CSR32, row_ptr=row_ptr.astype(np.int32), col=col.astype(np.int32),
                   val=np.ascontiguousarray(val, dtype=np.float64), n_csr=n, name=f"sdd_{n}")


def random_sdd_csr_scipy(n: int, seed: int = 0, nnz_lo: int = 7, nnz_hi: int = 27, margin: float = 1e-2) -> Problem:
    """The same matrix assembled with scipy.sparse (slow; a cross-check of random_sdd_csr)."""
    import scipy.sparse as sp
    rows, cols, vals = _sdd_draws(n, seed, nnz_lo, nnz_hi)
    U = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    A = (U + U.T).tocsr()
    A.sum_duplicates()
    diag = (1.0 + margin) * np.asarray(np.abs(A).sum(axis=1)).ravel()
    diag[diag == 0] = 1.0
    A = (A + sp.diags(diag)).tocsr()
    A.sort_indices()
    return Problem(CSR32, row_ptr=A.indptr.astype(np.int32), col=A.indices.astype(np.int32),
                   val=A.data.astype(np.float64), n_csr=n, name=f"sdd_{n}")


def laplacian_rhs(p: Problem, xstar: np.ndarray) -> np.ndarray:
    """b = A x* for a constant-coefficient Laplacian and dyadic x* (see module doc).

    Every intermediate is exact in binary64 (|x*| <= 1 on the 2^-30 grid, at most
    7 terms), so the result does not depend on evaluation order."""
    assert p.constant and p.layout in (STENCIL5_2D, STENCIL7_3D)
    scaled = xstar * (2.0 ** DYADIC_BITS)
    assert np.all(scaled == np.round(scaled)) and np.all(np.abs(xstar) <= 1.0), "x* must be dyadic"
    shape = (p.nz, p.ny, p.nx) if p.is_3d else (p.ny, p.nx)
    x = xstar.reshape(shape)
    b = (6.0 if p.is_3d else 4.0) * x
    for axis in range(x.ndim):
        sl_a = [slice(None)] * x.ndim
        sl_b = [slice(None)] * x.ndim
        sl_a[axis] = slice(1, None)
        sl_b[axis] = slice(0, -1)
        b[tuple(sl_a)] -= x[tuple(sl_b)]
        b[tuple(sl_b)] -= x[tuple(sl_a)]
    return np.ascontiguousarray(b.ravel())


# ---- the named workloads --------------------------------------------------

def poisson2d_manufactured(nx: int = 100, seed: int = 0):
    """2D 5-point Poisson, x* ~ U[-1,1] (dyadic, seed), b = A x*, x0 = 0."""
    p = laplacian_2d(nx)
    xs = dyadic_uniform_pm1(seed, p.n)
    return p, laplacian_rhs(p, xs), xs


def poisson3d_manufactured(n: int = 256, seed: int = 0):
    """3D 7-point Poisson on n^3, x* ~ U[-1,1] (dyadic, seed), b = A x*, x0 = 0."""
    p = laplacian_3d(n)
    xs = dyadic_uniform_pm1(seed, p.n)
    return p, laplacian_rhs(p, xs), xs


def poisson3d_manufactured_slab(nx: int, ny: int, nz: int, k0: int, k1: int, seed: int = 0) -> np.ndarray:
    """b = A x* on planes [k0, k1) of the nx x ny x nz Laplacian with the dyadic x* of
    seed (the values the whole-grid laplacian_rhs gives there, bit for bit: every term
    is exact), computed from x* on those planes and one plane on each side."""
    lo, hi = max(k0 - 1, 0), min(k1 + 1, nz)
    plane = nx * ny
    x = dyadic_uniform_pm1(seed, (hi - lo) * plane, offset=lo * plane).reshape(hi - lo, ny, nx)
    b = 6.0 * x
    b[1:] -= x[:-1]
    b[:-1] -= x[1:]
    b[:, 1:] -= x[:, :-1]
    b[:, :-1] -= x[:, 1:]
    b[:, :, 1:] -= x[:, :, :-1]
    b[:, :, :-1] -= x[:, :, 1:]
    return np.ascontiguousarray(b[k0 - lo:k0 - lo + (k1 - k0)].reshape(-1))


def lapl200():
    """The paper's lapl200 test case (Table 1): 200x200 unscaled 5-point Laplacian,
    b_j = 1/sqrt(n), x0 = 0."""
    p = laplacian_2d(200)
    return p, np.full(p.n, 1.0 / np.sqrt(p.n))

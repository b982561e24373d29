"""The seeded input generators (synthetic/): the random SDD CSR matrices of the serving
workload are assembled with torch (on a GPU when present) and must have the same bits as
the plain numpy reference, the same pattern as a scipy.sparse assembly of the same draws,
and strict diagonal dominance."""
import numpy as np
import pytest

import synthetic as S


@pytest.mark.parametrize("n,seed", [(2, 1), (97, 3), (5003, 4), (60000, 5)])
def test_random_sdd_csr_bits_and_structure(n, seed):
    a = S.random_sdd_csr(n, seed=seed)
    b = S.random_sdd_csr_numpy(n, seed=seed)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col) and np.array_equal(a.val, b.val)
    c = S.random_sdd_csr_scipy(n, seed=seed)
    assert np.array_equal(a.row_ptr, c.row_ptr) and np.array_equal(a.col, c.col)
    assert np.allclose(a.val, c.val, rtol=4e-15, atol=0)
    rows = np.repeat(np.arange(n), np.diff(a.row_ptr))
    on = a.col == rows
    assert np.all(np.bincount(rows[on], minlength=n) == 1)            # one diagonal entry per row
    off = np.zeros(n)
    np.add.at(off, rows[~on], np.abs(a.val[~on]))
    assert np.all(a.val[on] > off) and np.all(a.val[~on] <= 0)        # strictly diagonally dominant
    same_row = rows[1:] == rows[:-1]
    assert np.all(np.diff(a.col)[same_row] > 0)                       # sorted, duplicates merged
    # symmetric: the transpose has the same entries
    import scipy.sparse as sp
    A = sp.csr_matrix((a.val, a.col, a.row_ptr), shape=(n, n))
    assert abs(A - A.T).max() == 0.0


@pytest.mark.gpu
def test_random_sdd_csr_on_gpu_matches_numpy():
    import torch
    assert torch.cuda.is_available()
    a = S.random_sdd_csr(300001, seed=11)        # assembled on the GPU
    b = S.random_sdd_csr_numpy(300001, seed=11)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col) and np.array_equal(a.val, b.val)


def test_manufactured_slab_rhs_is_the_whole_grids():
    """The slab-local b = A x* of a z-slab has the bits of the whole grid's b there."""
    P, b, xs = S.poisson3d_manufactured(16)
    for k0, k1 in ((0, 5), (5, 11), (11, 16), (0, 16), (7, 8)):
        assert np.array_equal(S.poisson3d_manufactured_slab(16, 16, 16, k0, k1), b[k0 * 256:k1 * 256])

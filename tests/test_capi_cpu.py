"""The C-ABI library builds, loads and exports every symbol include/pcg.h declares;
argument checks that run before any CUDA call behave as documented (CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pcg.h")


@pytest.fixture(scope="module")
def libpath():
    from paper_1706_05988_gb300 import build
    return build.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(pcg_[a-z_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pcg_create", "pcg_solve", "pcg_solve_device", "pcg_destroy", "pcg_select_sigma",
                     "pcg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.check_output(["nm", "-D", "--defined-only", libpath]).decode()
    exported = set(re.findall(r"\sT\s(pcg_[a-z_]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert getattr(lib, n) is not None


def test_header_compiles_as_c(tmp_path):
    c = tmp_path / "t.c"
    c.write_text('#include "pcg.h"\nint main(void){pcg_result r; pcg_matrix m; (void)r; (void)m; return 0;}\n')
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), "-c", str(c),
                           "-o", str(tmp_path / "t.o")])


def test_argument_errors_without_gpu(libpath):
    from paper_1706_05988_gb300 import pcg as B
    L = B.lib()
    assert "libpcg" in B.pcg_version()
    out = ctypes.c_void_p(1)
    assert L.pcg_create(None, 0, ctypes.byref(out)) == B.PCG_EINVAL and out.value is None
    m = B.pcg_matrix()
    m.layout = 7
    assert L.pcg_create(ctypes.byref(m), 0, ctypes.byref(out)) == B.PCG_EINVAL
    m.layout = B.PCG_STENCIL5_2D
    m.nx, m.ny, m.nz = 0, 4, 1
    assert L.pcg_create(ctypes.byref(m), 0, ctypes.byref(out)) == B.PCG_EINVAL
    m.nx, m.ny, m.nz = 1 << 16, 1 << 16, 1
    assert L.pcg_create(ctypes.byref(m), 0, ctypes.byref(out)) == B.PCG_EINVAL      # beyond int32 indexing
    m.nx, m.ny = 4, 4
    assert L.pcg_create(ctypes.byref(m), 0x100, ctypes.byref(out)) == B.PCG_EINVAL  # unknown flag
    m.layout = B.PCG_CSR32
    m.n, m.nnz = 3, 2
    rp = (ctypes.c_int32 * 4)(0, 1, 1, 2)
    col = (ctypes.c_int32 * 2)(0, 5)                                                 # column out of range
    val = (ctypes.c_double * 2)(1.0, 1.0)
    m.row_ptr, m.col, m.val = ctypes.addressof(rp), ctypes.addressof(col), ctypes.addressof(val)
    assert L.pcg_create(ctypes.byref(m), 0, ctypes.byref(out)) == B.PCG_EINVAL
    assert L.pcg_solve(None, None, None, 2, 0.0, 0.0, 1, 0, None, None) == B.PCG_EINVAL
    assert L.pcg_select_sigma(None, None, 10, None, 1, None, None) == B.PCG_EINVAL
    assert L.pcg_kernel_stats(None, None, None, None) == B.PCG_EINVAL
    L.pcg_destroy(None)
    assert B.pcg_last_error(None) == "null context"


def test_argument_errors_of_the_extensions_without_gpu(libpath):
    """Jacobi / variable shift / batch / serving / self-check entry points reject bad arguments
    before touching the device."""
    from paper_1706_05988_gb300 import pcg as B
    L = B.lib()
    vp = ctypes.c_void_p
    assert L.pcg_set_shifts(None, None, 0) == B.PCG_EINVAL
    v = ctypes.c_double()
    assert L.pcg_get_param(None, B.PCG_PARAM_ITER_STAGES, ctypes.byref(v)) == B.PCG_EINVAL
    assert L.pcg_set_param(None, B.PCG_PARAM_ITER_STAGES, 2.0) == B.PCG_EINVAL
    assert L.pcg_psi_varsh(None, None, None, 10, None, 12, 1, None) == B.PCG_EINVAL
    assert L.pcg_batch_set_precision(None, B.PCG_MIXED_IR) == B.PCG_EINVAL
    assert L.pcg_batch_set_param(None, B.PCG_PARAM_MIXED_ETA, 0.5) == B.PCG_EINVAL
    assert L.pcg_batch_classes(None, None, None, None) == B.PCG_EINVAL
    assert L.pcg_batch_scalars(None, 4, None, None) == B.PCG_EINVAL
    assert L.pcg_batch_set_class_cluster(None, 0, 2) == B.PCG_EINVAL
    assert L.pcg_batch_set_class_occupancy(None, 0, 4) == B.PCG_EINVAL
    out = vp(1)
    assert L.pcg_batch_create(None, 1, 0, ctypes.byref(out)) == B.PCG_EINVAL
    m = B.pcg_matrix()
    m.layout = B.PCG_STENCIL5_2D
    m.nx, m.ny, m.nz = 8, 8, 1
    arr = (B.pcg_matrix * 1)(m)
    assert L.pcg_batch_create(ctypes.cast(arr, vp), 1, 0x4000, ctypes.byref(out)) == B.PCG_EINVAL
    t = ctypes.c_uint64()
    assert L.pcg_submit_ex(None, ctypes.byref(m), None, 1e-8, B.PCG_SPCG, 1.0, 10, 0, B.PCG_FP64,
                           ctypes.byref(t)) == B.PCG_EINVAL
    assert L.pcg_server_create(1024, 4, ctypes.byref(out)) == B.PCG_EINVAL       # budget below 1 MiB
    assert L.pcg_convert_check(None, None, None, None, -1) == B.PCG_EINVAL
    assert L.pcg_convert_check(None, None, None, None, 0) == B.PCG_OK


def test_csr_validation_over_several_chunks_without_gpu(libpath):
    """pcg_create checks a CSR matrix's row ranges and column indices in chunks of rows on
    several host threads: a valid matrix of many chunks passes to the device step (which
    fails without a GPU, as PCG_ECUDA or PCG_ENOMEM), and one bad entry anywhere, or a
    row range that runs backwards or past nnz, is PCG_EINVAL before any device call."""
    import numpy as np
    from paper_1706_05988_gb300 import pcg as B
    L = B.lib()
    n = 300_001                                           # five chunks of 65,536 rows, ragged tail
    deg = 3
    row_ptr = np.arange(0, deg * (n + 1), deg, dtype=np.int32)
    col = ((np.arange(n, dtype=np.int64)[:, None] + np.array([-1, 0, 1])) % n).astype(np.int32).ravel()
    val = np.tile(np.array([-1.0, 2.5, -1.0]), n)

    def create(rp, c, v):
        m = B.pcg_matrix()
        m.layout = B.PCG_CSR32
        m.n, m.nnz = n, int(rp[-1])
        m.row_ptr, m.col, m.val = rp.ctypes.data, c.ctypes.data, v.ctypes.data
        out = ctypes.c_void_p()
        s = L.pcg_create(ctypes.byref(m), 0, ctypes.byref(out))
        if s == B.PCG_OK:                                  # (run where a GPU is present)
            L.pcg_destroy(out)
        return s

    assert create(row_ptr, col, val) in (B.PCG_OK, B.PCG_ECUDA, B.PCG_ENOMEM)
    for k in (0, 3 * 65_536 + 7, col.size - 1):           # a bad column in the first, a middle, the last chunk
        bad = col.copy()
        bad[k] = n
        assert create(row_ptr, bad, val) == B.PCG_EINVAL
        bad[k] = -1
        assert create(row_ptr, bad, val) == B.PCG_EINVAL
    rp = row_ptr.copy()
    rp[200_000] = rp[200_001] + 1                          # a row range that runs backwards
    assert create(rp, col, val) == B.PCG_EINVAL
    rp = row_ptr.copy()
    rp[100_000] = int(row_ptr[-1]) + 5                     # past nnz (and backwards after it)
    assert create(rp, col, val) == B.PCG_EINVAL

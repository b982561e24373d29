"""Shifted pipelined Conjugate Gradients (arXiv 1706.05988) on one GB300.

The solver lives in libpcg.so (hand-written CUDA for sm_103a behind the C ABI
of include/pcg.h); `pcg` is its thin ctypes binding and `build` compiles it.
"""
from . import build  # noqa: F401
from .pcg import (METHODS, Batch, Server, PCG_CG, PCG_CSR32, PCG_DEVICE_PTRS, PCG_EBREAKDOWN, PCG_EINVAL, PCG_ENOTCONV, PCG_ENOTIMPL, PCG_ETIMEOUT,  # noqa: F401
                  PCG_FP64, PCG_MIXED_IR, PCG_OK, PCG_JACOBI, PCG_PCG, PCG_PERSISTENT, PCG_PROFILE, PCG_SPCG, PCG_STENCIL5_2D, PCG_STENCIL7_3D,
                  PCG_STENCIL_FP64_SUM, PCG_DOTS_SPLIT32, Matrix, pcg_apply,
                  PcgError, Solver, SolveResult, lib, pcg_create, pcg_destroy, pcg_kernel_stats,
                  pcg_kernel_stats_reset, pcg_last_error, pcg_psi, pcg_select_sigma, pcg_set_stream, pcg_solve,
                  pcg_set_param, pcg_get_param, pcg_set_shifts, pcg_psi_varsh, pcg_solve_device, pcg_version)

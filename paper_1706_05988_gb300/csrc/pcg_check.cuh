// Index checks of the checked build (compiled with -DPCG_CHECKED into libpcg_checked.so).
//
// The GPU's memory checker is not available here, so the kernels check the addresses they
// form themselves: every place that turns an index into a load or a store of a vector,
// a coefficient, a CSR entry, a halo plane or a bulk copy asks pcg_check(in bounds, code)
// first.  A failed check records its code in this translation unit's device word (the
// first failure wins) and the access is skipped -- the load reads 0, the store or copy is
// not issued -- so the kernel runs to its end and no barrier is left waiting.
// pcg_check_status (pcg_capi.cu) reads and clears the words of every translation unit.
// In ordinary builds pcg_check is the constant true and the checks compile away.
#pragma once
#include <cuda_runtime.h>

namespace pcgk {

// Codes of the checks (the first failure of a run is reported).
enum : unsigned {
  CHK_STENCIL_CENTRE = 1,   // a unit's own unknowns c0 .. c0+VEC-1 inside [0, n)
  CHK_STENCIL_Y = 2,        // the y neighbours' rows
  CHK_STENCIL_Z = 3,        // the z neighbours' planes
  CHK_STENCIL_X = 4,        // the x neighbours at the ends of a unit
  CHK_COEFF = 5,            // face coefficients of variable-coefficient stencils
  CHK_CSR_ROW = 6,          // a CSR row index and its row_ptr range
  CHK_CSR_COL = 7,          // a CSR column index
  CHK_BULK_COPY = 8,        // a bulk copy's global range, size and alignment
  CHK_SLAB_HALO = 9,        // a slab's halo plane
};

#ifdef PCG_CHECKED

// This translation unit's first failure code (0: none).
static __device__ unsigned int g_pcg_check_fail;

using CheckReader = unsigned (*)(bool clear);
void register_check_reader(CheckReader reader);   // pcg_capi.cu

namespace {
unsigned read_check_word(bool clear) {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_pcg_check_fail, sizeof v) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (clear && v != 0) {
    const unsigned z = 0;
    if (cudaMemcpyToSymbol(g_pcg_check_fail, &z, sizeof z) != cudaSuccess) cudaGetLastError();
  }
  return v;
}
struct CheckRegistrar {
  CheckRegistrar() { register_check_reader(&read_check_word); }
};
CheckRegistrar g_check_registrar;
}  // namespace

__device__ __forceinline__ bool pcg_check(bool ok, unsigned code) {
  if (!ok) atomicCAS(&g_pcg_check_fail, 0u, code);
  return ok;
}

#else

__device__ __forceinline__ constexpr bool pcg_check(bool, unsigned) { return true; }

#endif

}  // namespace pcgk

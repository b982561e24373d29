// binary32 <-> binary64 conversions on the integer pipe.
//
// On GB300 the hardware conversion instructions run at the FP64 pipe's rate
// (measured: 0.6 T conversions/s, the same as DFMA), and the mixed-precision
// kernels are bound by that pipe, so they convert with bit operations instead.
// Both functions are total: zeros, subnormals (inputs and results), overflow,
// Inf and NaN are handled with integer operations too, so no conversion
// instruction is ever issued (a rarely taken branch to the hardware conversion
// would still be issued, predicated off, on the FP64 pipe).  Every finite or
// infinite result equals the IEEE conversion (round to nearest even for
// double -> float); a NaN converts to a quiet NaN.
#pragma once
#include <cuda_runtime.h>

namespace pcgk {

// float -> double (exact).
__device__ __forceinline__ double f64_of(float f) {
  const unsigned u = (unsigned)__float_as_int(f);
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  const unsigned ex = (u >> 23) & 0xFFu;
  unsigned man = u & 0x7FFFFFu;
  unsigned long long bits;
  if (ex - 1u < 254u) {                            // normal
    bits = ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)man << 29);
  } else if (ex == 0u) {                           // zero or subnormal: normalise
    const int sh = __clz((int)man) - 8;            // moves the leading one to bit 23 (man != 0)
    const unsigned long long e64 = (unsigned long long)(897 - sh);
    bits = man ? (e64 << 52) | ((unsigned long long)((man << sh) & 0x7FFFFFu) << 29) : 0ull;
  } else {                                         // Inf, NaN (quieted)
    bits = (0x7FFull << 52) | ((unsigned long long)(man ? (man | 0x400000u) : 0u) << 29);
  }
  return __longlong_as_double((long long)(sign | bits));
}

// double -> float, round to nearest even.
__device__ __forceinline__ float f32_of(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(u >> 63) << 31;
  const int e = (int)(u >> 52) & 0x7FF;
  const unsigned long long m = u & 0x000FFFFFFFFFFFFFull;
  const int e32 = e - 896;
  unsigned bits;
  if (e == 0x7FF) {                                // Inf, NaN (quieted)
    bits = 0x7F800000u | (m ? 0x400000u | (unsigned)(m >> 29) : 0u);
  } else if (e32 >= 1) {                           // normal range (or overflow)
    const unsigned mant = (unsigned)(m >> 29);     // 23 stored bits
    const unsigned rem = (unsigned)(m & 0x1FFFFFFFull);
    bits = e32 >= 255 ? 0x7F800000u : (((unsigned)e32 << 23) | mant);
    if (e32 < 255 && (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u)))) ++bits;   // may carry to Inf
  } else if (e32 >= -24) {                         // subnormal result (or rounds up to the smallest normal)
    const unsigned long long full = m | (1ull << 52);
    const int sh = 30 - e32;                       // 30 .. 54
    const unsigned long long half = 1ull << (sh - 1);
    const unsigned long long rem = full & ((1ull << sh) - 1);
    bits = (unsigned)(full >> sh);
    if (rem > half || (rem == half && (bits & 1u))) ++bits;
  } else {                                         // below half the smallest subnormal: zero
    bits = 0u;
  }
  return __int_as_float((int)(sign | bits));
}

}  // namespace pcgk

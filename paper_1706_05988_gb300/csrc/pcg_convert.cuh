// binary32 <-> binary64 conversions on the integer pipe.
//
// On GB300 the hardware conversion instructions run at the FP64 pipe's rate
// (measured: 0.6 T conversions/s, the same as DFMA), so the mixed-precision
// kernels convert with bit operations instead.  Both functions handle normal
// numbers and zeros exactly like the IEEE conversion (round to nearest even
// for double -> float) and fall back to the hardware instruction for every
// other input (subnormal results or inputs, Inf, NaN, overflow), so the result
// is always bit-identical to a plain cast.
#pragma once
#include <cuda_runtime.h>

namespace pcgk {

// float -> double (exact).
__device__ __forceinline__ double f64_of(float f) {
  const unsigned u = (unsigned)__float_as_int(f);
  const unsigned mag = u & 0x7FFFFFFFu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if (mag - 0x00800000u < 0x7F000000u) {          // 1 <= exponent <= 254: normal
    return __longlong_as_double((long long)(sign | (((unsigned long long)mag + (896ull << 23)) << 29)));
  }
  if (mag == 0u) return __longlong_as_double((long long)sign);
  return (double)f;                                // subnormal, Inf, NaN
}

// double -> float, round to nearest even.
__device__ __forceinline__ float f32_of(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(u >> 63) << 31;
  const int e = (int)(u >> 52) & 0x7FF;
  const int e32 = e - 896;
  if (e32 >= 1 && e32 <= 254) {
    const unsigned long long m = u & 0x000FFFFFFFFFFFFFull;
    unsigned mant = (unsigned)(m >> 29);           // 23 stored bits
    const unsigned rem = (unsigned)(m & 0x1FFFFFFFull);
    unsigned bits = ((unsigned)e32 << 23) | mant;
    if (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) ++bits;   // carries into the exponent
    if (bits < 0x7F800000u) return __int_as_float((int)(sign | bits));
    return (float)d;                               // rounded up to overflow
  }
  if ((u << 1) == 0ull) return __int_as_float((int)sign);
  return (float)d;                                 // tiny, huge, Inf, NaN
}

}  // namespace pcgk

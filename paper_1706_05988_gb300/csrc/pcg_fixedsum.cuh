// Constant-coefficient Laplacian row  C*w_c - sum(neighbours)  (C = 6 in 3D, 4 in 2D)
// evaluated in 64-bit fixed point on the integer pipe and rounded once to binary64.
//
// Why: on GB300 the FP64 pipe issues 2 thread-instructions per cycle per SM while the
// integer pipe issues 64, so the five or six FP64 additions of a stencil row cost more
// FP64-pipe time than the rest of the fused iteration's FP64 work.
//
// How: every term is an integer significand times a power of two (C*w_c is exact: 6*m
// = 3*m * 2 and 4*m = m * 4).  All terms are aligned to the largest exponent E with
// kFxGuard guard bits below its unit in the last place and summed exactly in 64-bit
// integers (positive and negative terms apart; each sum stays below 2^62).  A term more than kFxGuard
// binades below E loses the bits shifted out (truncation, < 2^-kFxGuard ulp(2^E) per
// term).  The integer sum is then rounded to nearest-even binary64.
// Error: |result - exact| <= 0.5 ulp(result) + 6 * 2^-kFxGuard * ulp_E, where ulp_E is the
// unit in the last place of the largest term -- below the bound of any left-to-right
// FP64 summation of the same terms (which can reach several ulp_E).  The result is also
// independent of the order of the terms.
// Inf/NaN inputs or a result outside the normal binary64 range clear `ok`; the caller
// then evaluates the row with FP64 additions instead.
#pragma once
#include <cuda_runtime.h>

namespace pcgk {

constexpr int kFxGuard = 6;

struct FxRaw {
  unsigned long long mg;  // significand (implicit bit included for normal numbers) << kFxGuard
  int e;                  // biased exponent, 1 for zero and subnormals
  int neg;                // sign bit
  int special;            // Inf or NaN
};

struct FxTerm {
  unsigned long long mg;  // aligned significand before the exponent shift
  int e;
  int neg;
};

// Unpacks a binary64 value with integer operations only (an FP64 compare would
// use the FP64 pipe).
__device__ __forceinline__ FxRaw fx_raw(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int eb = (int)(u >> 52) & 0x7FF;
  FxRaw r;
  r.mg = ((u & 0x000FFFFFFFFFFFFFull) | ((unsigned long long)(eb != 0) << 52)) << kFxGuard;
  r.e = eb > 1 ? eb : 1;
  r.neg = (int)(u >> 63);
  r.special = eb == 0x7FF;
  return r;
}

// C * v as a term: C = 6 -> (3m, e+1); C = 4 -> (m, e+2).
template <int DIM>
__device__ __forceinline__ FxTerm fx_centre(const FxRaw& r) {
  FxTerm t;
  t.mg = DIM == 3 ? 3ull * r.mg : r.mg;
  t.e = r.e + (DIM == 3 ? 1 : 2);
  t.neg = r.neg;
  return t;
}

// -v as a term.
__device__ __forceinline__ FxTerm fx_minus(const FxRaw& r) {
  FxTerm t;
  t.mg = r.mg;
  t.e = r.e;
  t.neg = r.neg ^ 1;
  return t;
}

// Sum of the terms, rounded once.  Positive and negative terms go to separate
// accumulators (each below 2^62) and are aligned with one right shift each:
// (m << kFxGuard) >> d is m << (kFxGuard - d) exactly when d <= kFxGuard and
// truncates the bits below the accumulator's unit otherwise.
template <int NT>
__device__ __forceinline__ double fx_sum(const FxTerm (&t)[NT], bool& ok) {
  int E = t[0].e;
#pragma unroll
  for (int k = 1; k < NT; ++k) E = max(E, t[k].e);
  unsigned long long sp = 0ull, sn = 0ull;
#pragma unroll
  for (int k = 0; k < NT; ++k) {
    const unsigned long long a = t[k].mg >> min(E - t[k].e, 63);
    if (t[k].neg) {
      sn += a;
    } else {
      sp += a;
    }
  }
  if (sp == sn) return 0.0;
  const bool negative = sn > sp;
  const unsigned long long A = negative ? sn - sp : sp - sn;
  const int p = 63 - __clzll((long long)A);        // position of the leading one
  int er = p + E - kFxGuard - 52;                  // biased exponent of the result
  unsigned long long mant;
  if (p <= 52) {
    mant = A << (52 - p);
  } else {
    const int sh = p - 52;
    mant = A >> sh;
    const unsigned long long rem = A & ((1ull << sh) - 1ull);
    const unsigned long long half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) {
      ++mant;
      if (mant >> 53) {
        mant >>= 1;
        ++er;
      }
    }
  }
  ok = ok && er > 0 && er < 0x7FF;
  const unsigned long long sgn = negative ? (1ull << 63) : 0ull;
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(er & 0x7FF) << 52) |
                                          (mant & 0x000FFFFFFFFFFFFFull)));
}

}  // namespace pcgk

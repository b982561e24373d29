// Constant-coefficient Laplacian row  C*w_c - sum(neighbours)  (C = 6 in 3D, 4 in 2D)
// evaluated in 64-bit fixed point on the integer pipe and rounded once to binary64.
//
// Why: on GB300 the FP64 pipe issues 2 thread-instructions per cycle per SM while the
// integer pipe issues 64, so the five or six FP64 additions of a stencil row cost more
// FP64-pipe time than the rest of the fused iteration's FP64 work.
//
// How: every term is an integer significand times a power of two (C*w_c is exact: 6*m
// = 3*m * 2 and 4*m = m * 4).  All terms are aligned to the largest exponent E with
// kFxGuard guard bits below its unit in the last place and summed exactly in a signed
// 64-bit integer (the magnitudes bound the sum below 2^63).  A term more than kFxGuard
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
  unsigned long long m;   // significand (with the implicit bit for normal numbers)
  int e;                  // biased exponent, 1 for zero and subnormals
  int neg;                // sign bit
  int special;            // Inf or NaN
};

struct FxTerm {
  unsigned long long m;
  int e;
  int neg;
};

__device__ __forceinline__ FxRaw fx_raw(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int eb = (int)(u >> 52) & 0x7FF;
  FxRaw r;
  r.m = (u & 0x000FFFFFFFFFFFFFull) | ((unsigned long long)(eb != 0) << 52);
  r.e = eb > 1 ? eb : 1;
  r.neg = (int)(u >> 63);
  r.special = eb == 0x7FF;
  return r;
}

// C * v as a term: C = 6 -> (3m, e+1); C = 4 -> (m, e+2).
template <int DIM>
__device__ __forceinline__ FxTerm fx_centre(const FxRaw& r) {
  FxTerm t;
  t.m = DIM == 3 ? 3ull * r.m : r.m;
  t.e = r.e + (DIM == 3 ? 1 : 2);
  t.neg = r.neg;
  return t;
}

// -v as a term.
__device__ __forceinline__ FxTerm fx_minus(const FxRaw& r) {
  FxTerm t;
  t.m = r.m;
  t.e = r.e;
  t.neg = r.neg ^ 1;
  return t;
}

template <int NT>
__device__ __forceinline__ double fx_sum(const FxTerm (&t)[NT], bool& ok) {
  int E = t[0].e;
#pragma unroll
  for (int k = 1; k < NT; ++k) E = max(E, t[k].e);
  long long S = 0;
#pragma unroll
  for (int k = 0; k < NT; ++k) {
    const int d = E - t[k].e;
    unsigned long long a;
    if (d <= kFxGuard) {
      a = t[k].m << (kFxGuard - d);
    } else {
      const int sh = d - kFxGuard;
      a = sh < 64 ? (t[k].m >> sh) : 0ull;
    }
    S += t[k].neg ? -(long long)a : (long long)a;
  }
  if (S == 0) return 0.0;
  const unsigned long long sgn = S < 0 ? (1ull << 63) : 0ull;
  const unsigned long long A = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
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
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(er & 0x7FF) << 52) |
                                          (mant & 0x000FFFFFFFFFFFFFull)));
}

}  // namespace pcgk

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
// integers (positive and negative terms apart; each sum stays below 2^63).  A term more
// than kFxGuard binades below E loses the bits shifted out (truncation, < 2^-kFxGuard
// ulp(2^E) per term).  The integer sum is then rounded to nearest-even binary64.
// Error: |result - exact| <= 0.5 ulp(result) + 6 * 2^-kFxGuard * ulp_E, where ulp_E is the
// unit in the last place of the largest term -- below the bound of any left-to-right
// FP64 summation of the same terms (which can reach several ulp_E).  The result is also
// independent of the order of the terms.
//
// Two forms:
// - fx_sum (with fx_raw), for rows of finite terms whose result is a normal number; it
//   clears `ok` otherwise, and the caller evaluates that unit's rows with FP64 additions.
// - fx_sum_full (with fx_raw_full), for every row and with integer operations only: also
//   subnormal results (correctly rounded), overflow to infinity, and Inf/NaN terms, which
//   give what IEEE-754 addition gives in any order of the terms (NaN when a term is NaN or
//   infinities of both signs meet, else the infinity that is there).
// The 3D rows with two unknowns per thread use the first: the compiler branches over the
// FP64 fallback there, and the full form's extra instructions and registers cost 5 % of
// the sweep at 256^3.  The other stencils use the full form: for them the small FP64
// fallback was compiled into predicated instructions that still occupied the FP64 pipe
// when not taken (4 of 13 FP64 instructions per unknown of the 2D sweep, 6 of 15 of the
// 3D sweep with one unknown per thread), and the full form makes those sweeps 1.4-1.5x
// faster.
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
// accumulators (each below 2^63) and are aligned with one right shift each:
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

// ---------------------------------------------------------------- the full form

// Exponent given to Inf and NaN terms by fx_raw_full: above every finite term's (at most
// 0x7FE + 2), so a row holds one exactly when the largest exponent of its terms reaches
// it.  Their significand is 0 for an infinity and nonzero for a NaN.
constexpr int kFxSpecialE = 0x1000;

__device__ __forceinline__ FxTerm fx_raw_full(double v, int negate) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int eb = (int)(u >> 52) & 0x7FF;
  const unsigned long long frac = u & 0x000FFFFFFFFFFFFFull;
  FxTerm t;
  const bool special = eb == 0x7FF;
  t.mg = special ? (unsigned long long)(frac != 0ull) : (frac | ((unsigned long long)(eb != 0) << 52)) << kFxGuard;
  t.e = special ? kFxSpecialE : (eb > 1 ? eb : 1);
  t.neg = (int)(u >> 63) ^ negate;
  return t;
}

// The centre term C * v of fx_raw_full's terms (C = 6: (3m, e+1); C = 4: (m, e+2)).
template <int DIM>
__device__ __forceinline__ FxTerm fx_centre_full(double v) {
  FxTerm t = fx_raw_full(v, 0);
  t.mg = DIM == 3 ? 3ull * t.mg : t.mg;
  t.e += DIM == 3 ? 1 : 2;
  return t;
}

template <int NT>
__device__ __forceinline__ double fx_sum_full(const FxTerm (&t)[NT]) {
  int E = t[0].e;
#pragma unroll
  for (int k = 1; k < NT; ++k) E = max(E, t[k].e);
  unsigned long long sp = 0ull, sn = 0ull;
  // Inf and NaN terms (only when there are any): bit 0 a NaN, bit 1 +Inf, bit 2 -Inf
  int sc = 0;
  if (E >= kFxSpecialE) {
#pragma unroll
    for (int k = 0; k < NT; ++k)
      if (t[k].e >= kFxSpecialE) sc |= t[k].mg != 0ull ? 1 : (t[k].neg ? 4 : 2);
  }
#pragma unroll
  for (int k = 0; k < NT; ++k) {
    const unsigned long long a = t[k].mg >> min(E - t[k].e, 63);
    if (t[k].neg) {
      sn += a;
    } else {
      sp += a;
    }
  }
  const bool negative = sn > sp;
  const unsigned long long A = negative ? sn - sp : sp - sn;
  // The sum is worth A * 2^(E - 1075 - kFxGuard) (a term of biased exponent e and
  // significand M is worth M * 2^(e - 1075)).  It is rounded at bit sh of A: the bit
  // below the leading one's 52nd (a normal result), or the bit worth 2^-1074 when that
  // lies higher (a subnormal one).  m is then the result's significand, with the
  // implicit bit at 2^52 for a normal number, and the encoding is
  // (exponent field - 1) << 52 plus m: a rounding carry to 2^53, or to 2^52 from a
  // subnormal, moves into the exponent field by itself.
  const int p = 63 - __clzll((long long)(A | 1ull));   // position of the leading one
  const int sh = max(p - 52, kFxGuard + 1 - E);
  unsigned long long m;
  if (sh > 0) {
    m = A >> sh;
    const unsigned long long rem = A & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    m += rem > half || (rem == half && (m & 1ull)) ? 1ull : 0ull;
  } else {
    m = A << -sh;
  }
  const int ef = sh + E - kFxGuard - 1;                 // exponent field - 1 (>= 0)
  unsigned long long bits = ef + (int)(m >> 52) >= 0x7FF ? (0x7FFull << 52)   // overflow: infinity
                                                          : ((unsigned long long)ef << 52) + m;
  bits = A == 0ull ? 0ull : (bits | (negative ? (1ull << 63) : 0ull));
  if (sc != 0) {
    // the result IEEE-754 addition gives in any order: NaN with a NaN term or infinities
    // of both signs, else the infinity that is there
    bits = (sc & 1) || sc == 6 ? 0x7FF8000000000000ull : sc == 2 ? 0x7FF0000000000000ull : 0xFFF0000000000000ull;
  }
  return __longlong_as_double((long long)bits);
}

}  // namespace pcgk

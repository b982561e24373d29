// The merged dot products of the fused iteration, gamma_{i+1} = (r_{i+1}, r_{i+1}) and
// (w_{i+1}, r_{i+1}) (Algorithm 3, the dots of its reduction phase), accumulated on the
// FP32 pipe instead of the FP64 pipe.
//
// Why: GB300's FP64 pipe issues 2 thread-instructions per cycle per SM, the FP32 pipe 128
// and the integer pipe 64.  The fused iteration needs 7 FP64 fused multiply-adds per
// unknown for its vector recurrences; two more for the dots put its FP64 time (9 DFMA)
// at the time HBM needs to stream its 96 bytes.  The dots are sums, so they can be
// carried by an error-free float-float scheme.
// Measured (256^3 Laplacian, GB300): the FP64 pipe falls from 84 % to 63 % busy, but the
// sweep issues 27 % more instructions and waits longer on its global loads, and takes
// 0.34 ms against 0.29 ms with binary64 dots (0.32 ms with only (r, r) moved).  The form
// is therefore opt-in (PCG_DOTS_SPLIT32).
//
// How (each thread, over its units; then the usual binary64 block/grid reduction):
//  1. Each binary64 value v is scaled by 2^S and split with integer operations into two
//     binary32 values, v 2^S ~= h + l: h holds the leading 24 significant bits
//     (truncated), l the next 29 bits rounded to 24.  |v 2^S - (h + l)| <= 2^-49 |v 2^S|.
//  2. A product x y = (hx + lx)(hy + ly) is p + c: p = hx*hy rounded, e = fma(hx, hy, -p)
//     its exact error (TwoProd), and c = e + hx ly + lx hy + lx ly rounded (|c| <~ 2^-22 |p|).
//  3. The running sum is a pair (hi, lo): hi + p by TwoSum (exact: hi' + err = hi + p),
//     lo += err + c.
//  4. At the end the thread's sum is (double)hi + (double)lo, scaled back by 2^-S.
// Error per term: about 2^-47 |x y| (rounding of c and of lo); measured on p-CG vectors
// (24^3 Laplacian, iterations 0..60) 3e-15 for (r, r) and 1.5e-14 for (w, r) relative to
// the exact rational sums, against 1e-16..1e-15 for binary64 accumulation -- four orders
// below what alpha and beta parity needs.
//
// Range: S is chosen from the previous iteration's norms so that the scaled norm of each
// vector is below 2^kFfHeadroom.  Scaled entries below 2^-126 (their squares are below
// 2^-292 of the scaled sum) become 0.  Scaled entries must stay below 2^kFfMaxExp, so
// that a product stays below 2^112 and a thread's sum of up to 2^15 of them below the
// binary32 maximum.  A larger entry, or an Inf/NaN, sets `bad`; the thread then
// recomputes its dots in binary64 from the vectors it has just written (a rare branch,
// never taken while norms grow by less than 2^36 in one iteration).  A vector that
// shrinks by more than 2^140 in one iteration sums to 0 (an exact zero then stops the
// solve as converged).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace pcgk {

constexpr int kFfHeadroom = 20;   // log2 of the scaled norm bound
constexpr int kFfMaxExp = 56;     // log2 of the largest scaled entry taken on the FP32 pipe

struct FfSplit {
  float h, l;
};

// v 2^S as h + l (binary32), integer operations only.
__device__ __forceinline__ FfSplit ff_split(double v, int S, unsigned& bad) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned sign = hi & 0x80000000u;
  const int eb = (int)((hi >> 20) & 0x7FFu);
  const int e = eb - 1023 + 127 + S;                      // binary32 biased exponent of h
  const unsigned mh = ((hi & 0xFFFFFu) << 3) | (lo >> 29);  // 23 stored bits of h
  const unsigned R = lo & 0x1FFFFFFFu;                    // the 29 bits below h
  bad |= (unsigned)(eb == 0x7FF) | (unsigned)(eb != 0 && e >= 127 + kFfMaxExp);
  const bool hz = eb == 0 || e < 1;                       // zero, subnormal, or below binary32 range
  FfSplit s;
  s.h = __uint_as_float(hz ? 0u : (sign | ((unsigned)e << 23) | mh));
  // l: normalise R (leading one to bit 31), keep 24 bits, round to nearest on bit 7 (a
  // carry out of the mantissa field correctly increments the exponent field)
  const int lz = __clz(R);                                // 32 when R == 0
  const unsigned Rn = R << (lz & 31);
  const int el = e - 21 - lz;                             // biased exponent of R's leading one
  const unsigned lb = ((unsigned)el << 23) + ((Rn >> 8) & 0x7FFFFFu) + ((Rn >> 7) & 1u);
  s.l = __uint_as_float((hz || R == 0u || el < 1) ? 0u : (sign | lb));
  return s;
}

struct FfAcc {
  float hi = 0.0f, lo = 0.0f;
};

// a += p + c with p exact-split by TwoSum into a.hi; every operation is rounded as written
// (the _rn intrinsics keep the compiler from contracting or reassociating them).
__device__ __forceinline__ void ff_accumulate(FfAcc& a, float p, float c) {
  const float s = __fadd_rn(a.hi, p);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, __fadd_rn(err, c));
}

// a += x * y
__device__ __forceinline__ void ff_add_product(FfAcc& a, const FfSplit& x, const FfSplit& y) {
  const float p = __fmul_rn(x.h, y.h);
  float c = __fmaf_rn(x.h, y.h, -p);
  c = __fmaf_rn(x.h, y.l, c);
  c = __fmaf_rn(x.l, y.h, c);
  c = __fmaf_rn(x.l, y.l, c);
  ff_accumulate(a, p, c);
}

// a += x * x
__device__ __forceinline__ void ff_add_square(FfAcc& a, const FfSplit& x) {
  const float p = __fmul_rn(x.h, x.h);
  float c = __fmaf_rn(x.h, x.h, -p);
  c = __fmaf_rn(__fadd_rn(x.h, x.h), x.l, c);
  c = __fmaf_rn(x.l, x.l, c);
  ff_accumulate(a, p, c);
}

// (hi + lo) 2^-S in binary64
__device__ __forceinline__ double ff_value(const FfAcc& a, int S) {
  return scalbn((double)a.hi + (double)a.lo, -S);
}

// Scales for the next iteration from gamma = ||r||^2 and the Rayleigh-type estimate
// q = max(delta / gamma, sigma) of ||w|| / ||r|| (w ~ (A - sigma I) r): the scaled norms
// ||r|| 2^sr and q ||r|| 2^sw both lie below 2^kFfHeadroom.
__device__ __forceinline__ void ff_scales(double gamma, double delta, double sigma, int& sr, int& sw) {
  const int lr = gamma > 0.0 && isfinite(gamma) ? (ilogb(gamma) >> 1) + 1 : 0;   // ||r|| < 2^lr
  const double q = fmax(fabs(delta / gamma), sigma);
  const int lq = q > 0.0 && isfinite(q) ? ilogb(q) + 1 : 0;                      // q < 2^lq
  sr = max(-2000, min(2000, kFfHeadroom - lr));
  sw = max(-2000, min(2000, sr - lq));
}

}  // namespace pcgk

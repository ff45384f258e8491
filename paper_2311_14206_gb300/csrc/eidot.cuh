// Exact fixed-point dot products on the integer pipe.
//
// FP64 arithmetic on this GPU issues one warp instruction per ~16 cycles per
// SM, while 32-bit integer multiply-add issues at 64 lanes per cycle.  A dot
// product of FP64 vectors is therefore computed here as an exact integer sum:
// every operand x is rounded to a 52-bit signed integer X relative to a
// power-of-two scale shared by its vector (x ~ X * 2^(e-51), e the exponent of
// the vector's largest magnitude), X is split as X = hi * 2^26 + lo with
// |hi| <= 2^25 and 0 <= lo < 2^26, and the four partial products are summed
// exactly in three 64-bit accumulators (one IMAD.WIDE each).  The 128-bit
// result is rounded once to FP64.  The only rounding is the initial one of
// each operand (half a unit in 2^-51 of its vector's maximum) and the final
// one; the sum itself is exact and independent of summation order.
//
// Sums of up to 2048 terms stay within the accumulators' ranges.
#pragma once
#include "sdr_common.cuh"

namespace sdr {

struct __align__(8) Q52 {
  int hi;
  unsigned lo;
};

// Biased exponent field of |x| (0 for zero/subnormal).
__device__ __forceinline__ int bexp(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF);
}

// X = round(x * 2^delta * 2^(51 - e)), e = emax - 1022 where emax is the biased
// exponent of the largest |x * 2^delta| of the vector.  Integer operations only.
__device__ __forceinline__ Q52 q52(double x, int emax, int delta) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  const int sh = emax + 2 - (ex + delta);  // >= 2 for every element of the vector
  long long v = 0;
  if (ex != 0 && sh < 60) {
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const unsigned long long q = (mant + (1ull << (sh - 1))) >> sh;
    v = (b >> 63) ? -(long long)q : (long long)q;
  }
  Q52 r;
  r.hi = (int)(v >> 26);
  r.lo = (unsigned)(v & 0x3FFFFFFll);
  return r;
}

struct Acc3 {
  long long hh, mx, my;  // mx, my: the two mixed products in separate chains
  unsigned long long ll;
  __device__ __forceinline__ void zero() { hh = 0; mx = 0; my = 0; ll = 0ull; }
  // four 32 x 32 -> 64-bit multiply-adds (mad.wide), one per partial product
  __device__ __forceinline__ void mac(Q52 a, Q52 b) {
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(hh) : "r"(a.hi), "r"(b.hi));
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(mx) : "r"(a.hi), "r"((int)b.lo));
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(my) : "r"((int)a.lo), "r"(b.hi));
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(ll) : "r"(a.lo), "r"(b.lo));
  }
};

// Signed 128-bit (hi:lo) times 2^scale_exp, rounded to nearest even, with
// integer operations only (ldexp only when the exponent leaves the normal range).
__device__ __forceinline__ double i128_to_double(unsigned long long lo, unsigned long long hi, int scale_exp) {
  const bool neg = (long long)hi < 0;
  if (neg) {
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  if (hi == 0ull && lo == 0ull) return 0.0;
  const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
  const int msb = 127 - lz;
  unsigned long long mant;
  int e = msb;
  if (msb <= 52) {
    mant = lo << (52 - msb);
  } else {
    const int sh = msb - 52;  // 1 .. 75
    unsigned long long rb, sticky;
    if (sh < 64) {
      mant = (lo >> sh) | (sh ? (hi << (64 - sh)) : 0ull);
      rb = (lo >> (sh - 1)) & 1ull;
      sticky = (sh >= 2) ? (lo & ((1ull << (sh - 1)) - 1ull)) : 0ull;
    } else {
      const int s2 = sh - 64;
      mant = hi >> s2;
      rb = (s2 == 0) ? (lo >> 63) : ((hi >> (s2 - 1)) & 1ull);
      sticky = (s2 == 0) ? (lo & 0x7FFFFFFFFFFFFFFFull) : ((hi & ((1ull << (s2 - 1)) - 1ull)) | lo);
    }
    mant &= (1ull << 53) - 1ull;
    if (rb && (sticky || (mant & 1ull))) {
      mant += 1ull;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        e += 1;
      }
    }
  }
  const int be = e + scale_exp + 1023;
  double r;
  if (be > 0 && be < 2047) {
    r = __longlong_as_double((long long)(((unsigned long long)be << 52) | (mant & 0xFFFFFFFFFFFFFull)));
  } else {
    r = ldexp((double)mant, e - 52 + scale_exp);
  }
  return neg ? -r : r;
}

// Value of the accumulators times 2^scale_exp.
__device__ __forceinline__ double acc_to_double(const Acc3& a, int scale_exp) {
  unsigned long long lo = a.ll, hi = 0ull;
  add_shifted128(lo, hi, a.mx, 26);
  add_shifted128(lo, hi, a.my, 26);
  add_shifted128(lo, hi, a.hh, 52);
  return i128_to_double(lo, hi, scale_exp);
}

}  // namespace sdr

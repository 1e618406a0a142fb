// Integer helpers of the FP64-accurate Lanczos path (dtype ED_F64).
//
// GB300 runs FP64 arithmetic at about 1/70 of its FP32 rate, so a Lanczos vector of the
// FP64 path is stored as int64 fixed point: f = s * X with one FP64 scale s per vector and
// |X_i| <= 2^VB. Hop sums of H.v are then exact int64 additions; the few products with
// run-time scalars (t, U, a_j, b_j) are 64x64 -> 128-bit integer products rounded once per
// element; dot products and norms are accumulated exactly in 192-bit integers and rounded
// once to FP64 per step. No FP64 instruction runs per vector element.
#pragma once

#include <stdint.h>

namespace ed {

typedef __int128 i128;
typedef unsigned __int128 u128;

// Signed 192-bit accumulator (two's complement): value = hi * 2^128 + lo.
struct I192 {
  u128 lo;
  long long hi;
};

__device__ __forceinline__ void i192_zero(I192& a) {
  a.lo = 0;
  a.hi = 0;
}

__device__ __forceinline__ void i192_add(I192& a, i128 p) {
  const u128 u = (u128)p;
  const u128 s = a.lo + u;
  a.hi += (long long)(s < a.lo) + (p < 0 ? -1LL : 0LL);
  a.lo = s;
}

__device__ __forceinline__ void i192_add(I192& a, const I192& b) {
  const u128 s = a.lo + b.lo;
  a.hi += b.hi + (long long)(s < a.lo);
  a.lo = s;
}

__device__ __forceinline__ I192 i192_shfl_down(const I192& a, int off) {
  I192 r;
  const unsigned long long l0 = (unsigned long long)a.lo, l1 = (unsigned long long)(a.lo >> 64);
  const unsigned long long r0 = __shfl_down_sync(0xffffffffu, l0, off);
  const unsigned long long r1 = __shfl_down_sync(0xffffffffu, l1, off);
  r.lo = ((u128)r1 << 64) | (u128)r0;
  r.hi = __shfl_down_sync(0xffffffffu, a.hi, off);
  return r;
}

// Correctly rounded (nearest) conversion of the 192-bit integer to double.
__device__ __forceinline__ double i192_to_double(const I192& a) {
  const bool neg = a.hi < 0;
  unsigned long long w2 = (unsigned long long)a.hi;
  u128 lo = a.lo;
  if (neg) {  // magnitude = -a
    lo = ~lo + 1;
    w2 = ~w2 + (lo == 0 ? 1ull : 0ull);
  }
  const unsigned long long w1 = (unsigned long long)(lo >> 64), w0 = (unsigned long long)lo;
  unsigned long long top;
  bool sticky;
  int shift;  // value = top * 2^shift (+ sticky below)
  if (w2) {
    const int lz = __clzll(w2);
    top = lz ? (w2 << lz) | (w1 >> (64 - lz)) : w2;
    sticky = (lz ? (w1 << lz) != 0 : w1 != 0) || w0 != 0;
    shift = 128 - lz;
  } else if (w1) {
    const int lz = __clzll(w1);
    top = lz ? (w1 << lz) | (w0 >> (64 - lz)) : w1;
    sticky = lz ? (w0 << lz) != 0 : w0 != 0;
    shift = 64 - lz;
  } else {
    top = w0;
    sticky = false;
    shift = 0;
  }
  // fold the sticky bit into bit 0: the 11 discarded bits of `top` then round correctly
  const double m = __ull2double_rn(top | (sticky ? 1ull : 0ull));
  const double v = ldexp(m, shift);
  return neg ? -v : v;
}

// round(p * 2^k) for a 128-bit p, rounding half up; k may be negative (right shift) or
// non-negative (left shift; the caller guarantees no overflow).
__device__ __forceinline__ long long round_shift(i128 p, int k) {
  if (k >= 0) return (long long)(p << k);
  const int s = -k;
  if (s >= 127) return 0;
  const i128 half = (i128)1 << (s - 1);
  return (long long)((p + half) >> s);
}

// Coefficient c = m * 2^e with m an int64 mantissa, |m| < 2^62 for the largest of a set.
struct FxCoef {
  long long m;
  int e;
};

}  // namespace ed

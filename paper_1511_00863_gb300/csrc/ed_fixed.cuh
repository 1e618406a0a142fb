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

// The same arithmetic with the 128-bit words spelled out: 64 x 64 -> 128 products from the
// low and high halves of the multiply, sums as carry chains, and the rounding shift split on
// the (warp-uniform) shift amount. Results equal those of the i128 forms above bit for bit.
struct W128 {
  unsigned long long lo;
  long long hi;
};

__device__ __forceinline__ W128 smul128(long long a, long long b) {
  W128 r;
  r.lo = (unsigned long long)a * (unsigned long long)b;
  r.hi = __mul64hi(a, b);
  return r;
}

__device__ __forceinline__ W128 add128(const W128& a, const W128& b) {
  W128 r;
  asm("add.cc.u64 %0, %2, %4;\n\taddc.u64 %1, %3, %5;"
      : "=l"(r.lo), "=l"(r.hi)
      : "l"(a.lo), "l"(a.hi), "l"(b.lo), "l"(b.hi));
  return r;
}

// round_shift for a W128 value.
__device__ __forceinline__ long long round_shift128(const W128& p, int k) {
  if (k >= 0) return k >= 64 ? 0 : (long long)(p.lo << k);
  const int s = -k;
  if (s >= 127) return 0;
  if (s >= 64) {  // the half (2^(s-1)) reaches the high word only through bit 63 of the low one
    long long hi = p.hi;
    if (s == 64) {
      const unsigned long long l2 = p.lo + (1ull << 63);
      hi += (l2 < p.lo) ? 1 : 0;
    } else {
      hi += 1LL << (s - 65);
    }
    return hi >> (s - 64);
  }
  const unsigned long long l2 = p.lo + (1ull << (s - 1));
  const long long h2 = p.hi + ((l2 < p.lo) ? 1 : 0);
  return (long long)((l2 >> s) | ((unsigned long long)h2 << (64 - s)));
}

// 192-bit two's complement accumulator as three words (w2:w1:w0).
struct A192 {
  unsigned long long w0 = 0, w1 = 0, w2 = 0;
};

// a += x^2 with x = |v| < 2^64.
__device__ __forceinline__ void a192_add_sq(A192& a, unsigned long long x) {
  const unsigned long long lo = x * x, hi = __umul64hi(x, x);
  asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, 0;"
      : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2)
      : "l"(lo), "l"(hi));
}

// a += x y (signed).
__device__ __forceinline__ void a192_add_prod(A192& a, long long x, long long y) {
  const unsigned long long lo = (unsigned long long)x * (unsigned long long)y;
  const long long hi = __mul64hi(x, y);
  const unsigned long long ext = (unsigned long long)(hi >> 63);
  asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, %5;"
      : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2)
      : "l"(lo), "l"((unsigned long long)hi), "l"(ext));
}

__device__ __forceinline__ I192 a192_get(const A192& a) {
  I192 r;
  r.lo = ((u128)a.w1 << 64) | (u128)a.w0;
  r.hi = (long long)a.w2;
  return r;
}

// Coefficient c = m * 2^e with m an int64 mantissa, |m| < 2^62 for the largest of a set.
struct FxCoef {
  long long m;
  int e;
};

}  // namespace ed

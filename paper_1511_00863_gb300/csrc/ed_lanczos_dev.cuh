// Device helpers shared by the Lanczos drivers: lowest eigenvalue of T_j (Sec. 2.2) by
// Sturm-sequence bisection in FP64 and the per-step bookkeeping of b_{j+1}, breakdown and
// convergence.
#pragma once

#include "ed_internal.cuh"

namespace ed {

constexpr int kRedThreads = 256;
constexpr double kBreakdownRel = 1e-13;

// ------------------------------------------------------------------ Sturm bisection
// Number of eigenvalues of T_m below x (aa: 1-based diagonal a_1..a_m, bb: bb[i] = b_i^2 for
// i = 2..m, bb[1] = 0) = number of sign changes in the Sturm sequence p_0 = 1,
// p_i = (a_i - x) p_{i-1} - b_i^2 p_{i-2} (p_i = det of the leading i x i block of T - x I).
// The pair (p_{i-1}, p_i) is rescaled by exact powers of two to stay in range, so no division
// is needed. A vanishing p_i (a zero pivot p_i / p_{i-1}) is replaced by -2^-200 p_{i-1}, a
// tiny negative pivot. Signs are read from the bit patterns: two FP64 operations per row,
// which matters on GB300 where a warp-wide FP64 instruction occupies the pipe ~64x longer
// than an FP32 one.
__device__ __forceinline__ int sturm_count(const double* aa, const double* bb, int m, double x) {
  int cnt = 0;
  double p2 = 0.0, p1 = 1.0;
  unsigned long long s1 = 0ull;  // sign bit of p1
  for (int i = 1; i <= m; ++i) {
    double p = fma(aa[i] - x, p1, -bb[i] * p2);
    unsigned long long u = (unsigned long long)__double_as_longlong(p);
    if ((u << 1) == 0ull) {
      p = p1 * -0x1.0p-200;
      u = (unsigned long long)__double_as_longlong(p);
    }
    const unsigned long long sg = u & 0x8000000000000000ull;
    cnt += (int)((sg ^ s1) >> 63);
    s1 = sg;
    p2 = p1;
    p1 = p;
    const int e = (int)((u >> 52) & 0x7FF);
    if (e > 1023 + 400 || e < 1023 - 400) {  // keep |p| near 1: scale both by 2^-(e-1023)
      const int sh = 1023 - e;
      p1 = ldexp(p1, sh);
      p2 = ldexp(p2, sh);
    }
  }
  return cnt;
}

// ------------------------------------------------------------------ float-float Sturm count
// A value hi + lo of two FP32 numbers (about 48 significant bits), with the error-free
// transformations TwoSum (Knuth), FastTwoSum (Dekker 1971; |a| >= |b|) and the FMA product
// error (the product a b - fl(a b) is exact in one FMA). GB300 runs FP32 at about 64 times
// its FP64 rate, so the ~12 FP32 operations of one float-float operation still cost a few
// times less than one FP64 operation.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return FF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {
  const float s = a + b;
  return FF{s, b - (s - a)};
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
  const FF s = ff_two_sum(x.hi, y.hi);
  const FF t = ff_two_sum(x.lo, y.lo);
  const FF u = ff_fast_two_sum(s.hi, s.lo + t.hi);
  return ff_fast_two_sum(u.hi, u.lo + t.lo);
}
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ FF ff_of(double d) {
  const float hi = (float)d;
  return FF{hi, (float)(d - (double)hi)};
}

// sturm_count in float-float arithmetic (aa, bb as float-float copies of a_i and b_i^2). The
// count is exact for a tridiagonal whose entries differ from T's by a few units of 2^-48
// relative. The pair (p_{i-1}, p_i) is rescaled by powers of two to keep |p_i| within
// 2^-30..2^30 (FP32's range is narrow); a vanishing p_i becomes -2^-50 p_{i-1}.
__device__ __forceinline__ int sturm_count_ff(const FF* aa, const FF* bb, int m, FF x) {
  int cnt = 0;
  FF p2{0.f, 0.f}, p1{1.f, 0.f};
  bool n1 = false;
  const FF nx{-x.hi, -x.lo};
  for (int i = 1; i <= m; ++i) {
    const FF q = ff_mul(bb[i], p2);
    FF p = ff_add(ff_mul(ff_add(aa[i], nx), p1), FF{-q.hi, -q.lo});
    if (p.hi == 0.f) p = FF{-0x1.0p-50f * p1.hi, -0x1.0p-50f * p1.lo};  // (hi == 0 implies lo == 0)
    const bool n = p.hi < 0.f;
    cnt += n != n1 ? 1 : 0;
    n1 = n;
    p2 = p1;
    p1 = p;
    const int e = (int)((__float_as_uint(p1.hi) >> 23) & 0xFFu);
    if (e > 127 + 30 || e < 127 - 30) {
      const float sc = __uint_as_float((uint32_t)(254 - e) << 23);  // 2^(127 - e)
      p1 = FF{p1.hi * sc, p1.lo * sc};
      p2 = FF{p2.hi * sc, p2.lo * sc};
    }
  }
  return cnt;
}

// Two float-float counts at once (x0, x1): two independent recurrences interleaved, so a
// thread's dependent chain of FP32 operations hides its own latency.
__device__ __forceinline__ void sturm_count_ff2(const FF* aa, const FF* bb, int m, FF x0, FF x1,
                                                int& c0, int& c1) {
  c0 = 0;
  c1 = 0;
  FF p2a{0.f, 0.f}, p1a{1.f, 0.f}, p2b{0.f, 0.f}, p1b{1.f, 0.f};
  bool na = false, nb = false;
  const FF nx0{-x0.hi, -x0.lo}, nx1{-x1.hi, -x1.lo};
  for (int i = 1; i <= m; ++i) {
    const FF ai = aa[i], bi = bb[i];
    const FF qa = ff_mul(bi, p2a), qb = ff_mul(bi, p2b);
    FF pa = ff_add(ff_mul(ff_add(ai, nx0), p1a), FF{-qa.hi, -qa.lo});
    FF pb = ff_add(ff_mul(ff_add(ai, nx1), p1b), FF{-qb.hi, -qb.lo});
    if (pa.hi == 0.f) pa = FF{-0x1.0p-50f * p1a.hi, -0x1.0p-50f * p1a.lo};
    if (pb.hi == 0.f) pb = FF{-0x1.0p-50f * p1b.hi, -0x1.0p-50f * p1b.lo};
    const bool ma = pa.hi < 0.f, mb = pb.hi < 0.f;
    c0 += ma != na ? 1 : 0;
    c1 += mb != nb ? 1 : 0;
    na = ma;
    nb = mb;
    p2a = p1a;
    p1a = pa;
    p2b = p1b;
    p1b = pb;
    const int ea = (int)((__float_as_uint(p1a.hi) >> 23) & 0xFFu);
    if (ea > 127 + 30 || ea < 127 - 30) {
      const float sc = __uint_as_float((uint32_t)(254 - ea) << 23);
      p1a = FF{p1a.hi * sc, p1a.lo * sc};
      p2a = FF{p2a.hi * sc, p2a.lo * sc};
    }
    const int eb = (int)((__float_as_uint(p1b.hi) >> 23) & 0xFFu);
    if (eb > 127 + 30 || eb < 127 - 30) {
      const float sc = __uint_as_float((uint32_t)(254 - eb) << 23);
      p1b = FF{p1b.hi * sc, p1b.lo * sc};
      p2b = FF{p2b.hi * sc, p2b.lo * sc};
    }
  }
}

// Shared-memory workspace of sturm_lowest for T_m with m <= cap - 2: a_i and b_i^2 in FP64
// and as float-float pairs, 4 cap doubles (kSturmWork for any m <= ED_MAX_STEPS).
__host__ __device__ constexpr int sturm_work_doubles(int cap) { return 4 * cap; }
constexpr int kSturmCap = ED_MAX_STEPS + 2;
constexpr int kSturmWork = sturm_work_doubles(kSturmCap);

// lambda_min(T_m) by multisection, called by the whole block (>= 128 threads); returns the
// upper end of the final bracket (valid in every thread). a, b: 1-based a_1..a_m, b_2..b_m.
// The diagonal and the squared off-diagonal are staged in `work` (sturm_work_doubles(cap)
// doubles of shared memory, m <= cap - 2). Each round evaluates the Sturm count at 128 interior points of the bracket
// (four warps, one per SM sub-partition) and keeps the sub-interval holding the first
// eigenvalue. The rounds first count in float-float arithmetic, until the bracket is within
// delta = 2^-40 ||T|| (256 times the float-float count's backward error); the bracket is
// then widened by delta on both sides and FP64 rounds narrow it until it stops shrinking in
// FP64, so the result has the precision of an all-FP64 multisection at about half its FP64
// work. With a hint (a previous lambda_min of a leading block of T_m, an upper bound by
// Cauchy interlacing; NaN = none), a first round probes geometrically spaced points below
// it, so a bracket of the size of the last change is found in one round.
__device__ __forceinline__ double sturm_lowest(const double* a, const double* b, int m,
                                               double hint, double* work, int cap = kSturmCap) {
  constexpr int P = 128;
  double* aa = work;
  double* bb = work + cap;
  FF* af = reinterpret_cast<FF*>(work + 2 * cap);
  FF* bf = af + cap;
  __shared__ double lo_s, hi_s, delta_s;
  __shared__ double glo_s[32], ghi_s[32];
  __shared__ int first_s, last0_s, top_s;
  // staging and the Gershgorin bounds, one row per thread (a serial pass over the rows costs
  // about 10 us at m = 56 on GB300's FP64 pipe)
  double glo = INFINITY, ghi = -INFINITY;
  for (int i = 1 + threadIdx.x; i <= m; i += blockDim.x) {
    const double ai = a[i];
    aa[i] = ai;
    bb[i] = i > 1 ? b[i] * b[i] : 0.0;
    af[i] = ff_of(ai);
    bf[i] = ff_of(bb[i]);
    const double r = (i > 1 ? fabs(b[i]) : 0.0) + (i < m ? fabs(b[i + 1]) : 0.0);
    glo = fmin(glo, ai - r);
    ghi = fmax(ghi, ai + r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    glo_s[threadIdx.x >> 5] = glo;
    ghi_s[threadIdx.x >> 5] = ghi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double lo = INFINITY, hi = -INFINITY;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) {
      lo = fmin(lo, glo_s[w]);
      hi = fmax(hi, ghi_s[w]);
    }
    const double span = fmax(fmax(fabs(lo), fabs(hi)), 1e-300);
    lo_s = lo - 1e-15 * span - 1e-300;
    hi_s = hi + 1e-15 * span + 1e-300;
    delta_s = 0x1.0p-40 * span;
    last0_s = -1;
    top_s = 0;
  }
  __syncthreads();
  const double delta = delta_s;
  // ---- probe round below the hint (float-float counts, down to delta below it)
  if (isfinite(hint)) {
    const double lo = lo_s;
    const double hi = fmin(hi_s, hint + 1e-14 * fmax(fabs(hint), 1e-300) + delta);
    const double D = hi - lo;
    const double tiny = delta;
    if (D > 2.0 * tiny) {
      // x_i = hi - D r^i, i = 0..P-2 (x_0 = lo), r^(P-2) = tiny / D; lane P-1 checks x = hi
      const double lr = log2(tiny / D) / (double)(P - 2);
      if (threadIdx.x < P) {
        const int i = threadIdx.x;
        const double x = (i == P - 1) ? hi : hi - D * exp2(lr * (double)i);
        const int c = (x > lo && x <= hi) ? sturm_count_ff(af, bf, m, ff_of(x)) : (x <= lo ? 0 : 1);
        if (i == P - 1) {
          top_s = c;
        } else if (c == 0) {
          atomicMax(&last0_s, i);
        }
      }
      __syncthreads();
      if (threadIdx.x == 0 && top_s >= 1) {
        const int k = last0_s;  // largest probe index still below lambda_min
        if (k >= 0) {
          const double nlo = hi - D * exp2(lr * (double)k);
          const double nhi = (k + 1 <= P - 2) ? hi - D * exp2(lr * (double)(k + 1)) : hi;
          lo_s = fmax(nlo, lo);
          hi_s = fmin(nhi, hi);
        } else {
          hi_s = hi;
        }
      }
      __syncthreads();
    }
  }
  // ---- equally spaced rounds: float-float (2 P points, two per thread) while the bracket is
  // wider than 4 delta, then (after widening by delta) FP64 (P points) until the bracket is
  // within 4 units in the last place of its ends or stops shrinking
  bool fp64 = false;
  for (int round = 0; round < 160; ++round) {
    if (!fp64 && !(hi_s - lo_s > 4.0 * delta)) {
      fp64 = true;
      __syncthreads();
      if (threadIdx.x == 0) {
        lo_s -= delta;
        hi_s += delta;
      }
      __syncthreads();
    }
    const int np = fp64 ? P : 2 * P;
    const double lo = lo_s, hi = hi_s;
    const double w = (hi - lo) / (double)(np + 1);
    if (threadIdx.x == 0) first_s = np;
    __syncthreads();
    if (threadIdx.x < P) {
      if (fp64) {
        const double x = lo + w * (double)(threadIdx.x + 1);
        if (x > lo && x < hi && sturm_count(aa, bb, m, x) >= 1) atomicMin(&first_s, (int)threadIdx.x);
      } else {
        const int k0 = threadIdx.x, k1 = threadIdx.x + P;
        const double x0 = lo + w * (double)(k0 + 1), x1 = lo + w * (double)(k1 + 1);
        int c0, c1;
        sturm_count_ff2(af, bf, m, ff_of(x0), ff_of(x1), c0, c1);
        if (x0 > lo && x0 < hi && c0 >= 1) atomicMin(&first_s, k0);
        else if (x1 > lo && x1 < hi && c1 >= 1) atomicMin(&first_s, k1);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const int k = first_s;
      const double nhi = (k < np) ? lo + w * (double)(k + 1) : hi;
      const double nlo = (k > 0) ? lo + w * (double)k : lo;
      lo_s = fmax(nlo, lo);
      hi_s = fmin(nhi, hi);
    }
    __syncthreads();
    if (fp64) {
      if (!(lo_s < hi_s) || (lo_s == lo && hi_s == hi)) break;
      const double mid = 0.5 * (lo_s + hi_s);
      if (!(mid > lo_s && mid < hi_s)) break;
      const double mag = fmax(fabs(lo_s), fabs(hi_s));
      if (hi_s - lo_s <= 4.0 * (mag > 0.0 ? ldexp(1.0, ilogb(mag) - 52) : 0.0)) break;
    }
  }
  return hi_s;
}

// Eigenvector y of T_m (a: a_1..a_m, b: b_2..b_m, 1-based; b[m + 1] is read as the scale
// bound's last term) for its lowest eigenvalue lam, by inverse iteration: three solves of
// (T - sigma I) z = y with sigma just below lam, where T - sigma I is positive definite, so
// the tridiagonal LU without pivoting is stable. The LU factors (pivot reciprocals) are
// formed once and reused by the three solves: m divisions in all, which matters for one
// thread at GB300's FP64 rate. One thread; y[1..m] normalised; work holds 2 (m + 2) doubles.
__device__ __forceinline__ void tridiag_ritz_vector(const double* a, const double* b, int m,
                                                    double lam, double* y, double* work) {
  double scale = fabs(lam);
  for (int i = 1; i <= m; ++i) scale = fmax(scale, fabs(a[i]) + b[i] + b[i + 1]);
  const double sigma = lam - 1e-10 * fmax(scale, 1e-300);
  double* inv = work;            // reciprocals of the pivots
  double* z = work + (m + 2);    // right-hand side / solution
  inv[1] = 1.0 / (a[1] - sigma);
  for (int i = 2; i <= m; ++i) inv[i] = 1.0 / ((a[i] - sigma) - b[i] * b[i] * inv[i - 1]);
  for (int i = 1; i <= m; ++i) y[i] = 1.0;
  for (int it = 0; it < 3; ++it) {
    // forward elimination, then back substitution, of (T - sigma I) z = y
    z[1] = y[1];
    for (int i = 2; i <= m; ++i) z[i] = y[i] - b[i] * inv[i - 1] * z[i - 1];
    z[m] *= inv[m];
    for (int i = m - 1; i >= 1; --i) z[i] = (z[i] - b[i + 1] * z[i + 1]) * inv[i];
    double nrm = 0.0;
    for (int i = 1; i <= m; ++i) nrm = fma(z[i], z[i], nrm);
    const double r = 1.0 / sqrt(nrm);
    for (int i = 1; i <= m; ++i) y[i] = z[i] * r;
  }
}

// Thread 0 of the finish kernel: record b_{j+1}, update the breakdown scale, advance j.
// Returns 1 on breakdown (b_{j+1} <= 1e-13 max(1, max_i |a_i| + b_i)), else 0.
__device__ __forceinline__ int finish_record_beta(LzScalars* S, int j, double beta) {
  const double ts = fmax(S->tscale, fabs(S->alpha[j]) + S->beta[j]);
  S->tscale = ts;
  S->beta[j + 1] = beta;
  S->j = j;
  return (beta > kBreakdownRel * fmax(1.0, ts)) ? 0 : 1;
}

// Whole block: E0(j) = lambda_min(T_j) when due, convergence test, final status.
__device__ __forceinline__ void finish_tail(LzScalars* S, int j, int st) {
  __shared__ double sturm_work[kSturmWork];
  const bool check = st != 0 || j >= S->max_steps || (j % S->check_every) == 0;
  if (check) {
    const double E = sturm_lowest(S->alpha, S->beta, j, S->last_E0_step > 0 ? S->last_E0 : NAN,
                                  sturm_work);
    if (threadIdx.x == 0) {
      S->E0[j] = E;
      if (st == 0 && S->tol > 0.0 && S->last_E0_step > 0 &&
          fabs(E - S->last_E0) <= S->tol * fmax(fabs(E), 1.0))
        st = 2;
      S->last_E0 = E;
      S->last_E0_step = j;
    }
  }
  if (threadIdx.x == 0) {
    if (st == 0 && j >= S->max_steps) st = 3;
    S->status = st;
  }
}

}  // namespace ed

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

// Shared-memory workspace of sturm_lowest: a_i and b_i^2 for i <= ED_MAX_STEPS + 1.
constexpr int kSturmWork = 2 * (ED_MAX_STEPS + 2);

// lambda_min(T_m) by multisection, called by the whole block (>= 128 threads); returns the
// upper end of the final bracket (valid in every thread). a, b: 1-based a_1..a_m, b_2..b_m.
// The diagonal and the squared off-diagonal are staged in `work` (kSturmWork doubles of
// shared memory). Each round
// evaluates the Sturm count at 128 interior points of the bracket (four warps, one per SM
// sub-partition) and keeps the sub-interval holding the first eigenvalue, until the bracket
// stops shrinking in FP64. With a hint (a previous lambda_min of a leading block of T_m, an
// upper bound by Cauchy interlacing; NaN = none), a first round probes geometrically spaced
// points below it, so a bracket of the size of the last change is found in one round.
__device__ __forceinline__ double sturm_lowest(const double* a, const double* b, int m,
                                               double hint, double* work) {
  constexpr int P = 128;
  double* aa = work;
  double* bb = work + (ED_MAX_STEPS + 2);
  __shared__ double lo_s, hi_s;
  __shared__ int first_s, last0_s, top_s;
  for (int i = 1 + threadIdx.x; i <= m; i += blockDim.x) {
    aa[i] = a[i];
    bb[i] = i > 1 ? b[i] * b[i] : 0.0;
  }
  if (threadIdx.x == 0) {
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 1; i <= m; ++i) {
      const double r = (i > 1 ? fabs(b[i]) : 0.0) + (i < m ? fabs(b[i + 1]) : 0.0);
      lo = fmin(lo, a[i] - r);
      hi = fmax(hi, a[i] + r);
    }
    const double span = fmax(fmax(fabs(lo), fabs(hi)), 1e-300);
    lo_s = lo - 1e-15 * span - 1e-300;
    hi_s = hi + 1e-15 * span + 1e-300;
    last0_s = -1;
    top_s = 0;
  }
  __syncthreads();
  // ---- probe round below the hint
  if (isfinite(hint)) {
    const double lo = lo_s;
    const double hi = fmin(hi_s, hint + 1e-14 * fmax(fabs(hint), 1e-300));
    const double D = hi - lo;
    const double tiny = 1e-16 * fmax(fabs(hi), 1e-300);
    if (D > 2.0 * tiny) {
      // x_i = hi - D r^i, i = 0..P-2 (x_0 = lo), r^(P-2) = tiny / D; lane P-1 checks x = hi
      const double lr = log2(tiny / D) / (double)(P - 2);
      if (threadIdx.x < P) {
        const int i = threadIdx.x;
        const double x = (i == P - 1) ? hi : hi - D * exp2(lr * (double)i);
        const int c = (x > lo && x <= hi) ? sturm_count(aa, bb, m, x) : (x <= lo ? 0 : 1);
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
  // ---- equally spaced rounds
  for (int round = 0; round < 128; ++round) {
    const double lo = lo_s, hi = hi_s;
    const double w = (hi - lo) / (double)(P + 1);
    if (threadIdx.x == 0) first_s = P;
    __syncthreads();
    if (threadIdx.x < P) {
      const double x = lo + w * (double)(threadIdx.x + 1);
      const bool valid = x > lo && x < hi;
      if (valid && sturm_count(aa, bb, m, x) >= 1) atomicMin(&first_s, (int)threadIdx.x);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const int k = first_s;
      const double nhi = (k < P) ? lo + w * (double)(k + 1) : hi;
      const double nlo = (k > 0) ? lo + w * (double)k : lo;
      lo_s = fmax(nlo, lo);
      hi_s = fmin(nhi, hi);
    }
    __syncthreads();
    if (!(lo_s < hi_s) || (lo_s == lo && hi_s == hi)) break;
    const double mid = 0.5 * (lo_s + hi_s);
    if (!(mid > lo_s && mid < hi_s)) break;
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

// Device helpers shared by the Lanczos drivers: lowest eigenvalue of T_j (Sec. 2.2) by
// Sturm-sequence bisection in FP64 and the per-step bookkeeping of b_{j+1}, breakdown and
// convergence.
#pragma once

#include "ed_internal.cuh"

namespace ed {

constexpr int kRedThreads = 256;
constexpr double kBreakdownRel = 1e-13;

// ------------------------------------------------------------------ Sturm bisection
// Number of eigenvalues of T_m below x (a: 1-based diagonal a[1..m], b: b[2..m]) = number
// of sign changes in the Sturm sequence p_0 = 1, p_i = (a_i - x) p_{i-1} - b_i^2 p_{i-2}
// (p_i = det of the leading i x i block of T - x I). The pair (p_{i-1}, p_i) is rescaled by
// exact powers of two to stay in range, so no division is needed; a zero p_i is given the
// sign opposite to p_{i-1} (a vanishing pivot counted as negative).
__device__ __forceinline__ int sturm_count(const double* a, const double* b, int m, double x) {
  int cnt = 0;
  double p2 = 0.0, p1 = 1.0;
  for (int i = 1; i <= m; ++i) {
    const double b2 = (i > 1) ? b[i] * b[i] : 0.0;
    double p = fma(a[i] - x, p1, -b2 * p2);
    if (p == 0.0) p = p1 > 0.0 ? -0x1.0p-1000 : 0x1.0p-1000;
    cnt += (p < 0.0) != (p1 < 0.0);
    p2 = p1;
    p1 = p;
    const int e = (int)((__double_as_longlong(p1) >> 52) & 0x7FF);
    if (e > 1023 + 400 || e < 1023 - 400) {  // keep |p| near 1: scale both by 2^-(e-1023)
      const int sh = 1023 - e;
      p1 = ldexp(p1, sh);
      p2 = ldexp(p2, sh);
    }
  }
  return cnt;
}

// lambda_min(T_m) by multisection: each round evaluates the Sturm count at 32 interior
// points of the bracket (one warp; the FP64 work per round is what limits this on GB300) and
// keeps the sub-interval holding the first eigenvalue, until the bracket stops shrinking in
// FP64. Called by the whole block; returns the upper end (valid in every thread).
__device__ __forceinline__ double sturm_lowest(const double* a, const double* b, int m) {
  __shared__ double lo_s, hi_s;
  __shared__ int first_s;
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
  }
  __syncthreads();
  const int P = 32;
  for (int round = 0; round < 128; ++round) {
    const double lo = lo_s, hi = hi_s;
    const double w = (hi - lo) / (double)(P + 1);
    if (threadIdx.x == 0) first_s = P;
    __syncthreads();
    if (threadIdx.x < P) {
      const double x = lo + w * (double)(threadIdx.x + 1);
      const bool valid = x > lo && x < hi;
      if (valid && sturm_count(a, b, m, x) >= 1) atomicMin(&first_s, (int)threadIdx.x);
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
  const bool check = st != 0 || j >= S->max_steps || (j % S->check_every) == 0;
  if (check) {
    const double E = sturm_lowest(S->alpha, S->beta, j);
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

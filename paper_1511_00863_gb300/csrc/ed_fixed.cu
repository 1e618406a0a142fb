// FP64-accurate Lanczos (Sec. 2.2, Algorithm 1) with int64 fixed-point vectors.
//
// A vector is f = s * X (s: FP64 scale in LzScalars, X: int64, |X_i| <= 2^vb with
// vb = 62 - ceil(log2(hops + n_max + 2))), so that a hop sum of up to `hops` elements and
// the diagonal product n X never overflow. One step j on buffers cur (f_j) and prev
// (f_{j-1}):
//   plan   (1 thread):  choose W's scale s_w = s_cur 2^r so that |W| <= 2^(vb-1), and the
//                       integer coefficients of  W = round((a S + b n X + c P) 2^k)  with
//                       a 2^k = -t 2^-r, b 2^k = U 2^-r, c 2^k = -b_j (s_prev/s_cur) 2^-r;
//   H.v    (fused):     S = exact int64 hop sum (Sec. 4 Eqs. 5-6), P = X_prev, W written
//                       over P; partial sums of W X_cur exact in 192 bits;
//   update:             a_j = s_w s_cur sum(W X_cur) (one FP64 rounding),
//                       Q = W + round(d X_cur 2^k2) with d 2^k2 = -a_j s_cur / s_w,
//                       exact partial sums of Q^2 and max |Q|;
//   finish (1 CTA):     b_{j+1} = s_w sqrt(sum Q^2), f_{j+1} = (s_w / b_{j+1}) Q.
// Every element of every vector is rounded once per pass, to a grid of 2^-vb of the
// vector's current maximum; sums and dot products are exact.
#include <cmath>

#include "ed_fixed.cuh"
#include "ed_internal.cuh"
#include "ed_lanczos_dev.cuh"

namespace ed {

constexpr int kFxThreads = 256;

FxRun fx_make(const ed_basis* b) {
  FxRun f;
  f.hops = b->up.maxhops + b->dn.maxhops;
  f.nmax = b->n_up < b->n_dn ? b->n_up : b->n_dn;
  const int need = f.hops + f.nmax + 2;
  int hb = 0;
  while ((1 << hb) < need) ++hb;
  f.vb = 62 - hb;
  return f;
}

// ------------------------------------------------------------------ reductions
// Block reduction of a 192-bit sum and a max; thread 0 writes out[0..3] =
// (lo bits 0..63, lo bits 64..127, hi, max).
__device__ __forceinline__ void fx_block_reduce(I192 v, long long mx, long long* out) {
  __shared__ unsigned long long sm[32][4];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const I192 w = i192_shfl_down(v, o);
    i192_add(v, w);
    mx = max(mx, (long long)__shfl_down_sync(0xffffffffu, mx, o));
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) {
    sm[wid][0] = (unsigned long long)v.lo;
    sm[wid][1] = (unsigned long long)(v.lo >> 64);
    sm[wid][2] = (unsigned long long)v.hi;
    sm[wid][3] = (unsigned long long)mx;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    I192 a;
    i192_zero(a);
    long long m = 0;
    if (lane < nw) {
      a.lo = ((u128)sm[lane][1] << 64) | (u128)sm[lane][0];
      a.hi = (long long)sm[lane][2];
      m = (long long)sm[lane][3];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const I192 w = i192_shfl_down(a, o);
      i192_add(a, w);
      m = max(m, (long long)__shfl_down_sync(0xffffffffu, m, o));
    }
    if (lane == 0) {
      out[0] = (long long)(unsigned long long)a.lo;
      out[1] = (long long)(unsigned long long)(a.lo >> 64);
      out[2] = a.hi;
      out[3] = m;
    }
  }
  __syncthreads();
}

// Sum (exact) and max of n partial records of 4 words; every thread gets the result.
__device__ __forceinline__ void fx_sum_partials(const long long* __restrict__ p, int n, I192& sum,
                                                long long& mx) {
  __shared__ long long out[4];
  I192 v;
  i192_zero(v);
  long long m = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    I192 w;
    w.lo = ((u128)(unsigned long long)p[4 * i + 1] << 64) | (u128)(unsigned long long)p[4 * i];
    w.hi = p[4 * i + 2];
    i192_add(v, w);
    m = max(m, p[4 * i + 3]);
  }
  fx_block_reduce(v, m, out);
  sum.lo = ((u128)(unsigned long long)out[1] << 64) | (u128)(unsigned long long)out[0];
  sum.hi = out[2];
  mx = out[3];
  __syncthreads();
}

__device__ __forceinline__ long long sgn_apply(long long v, uint32_t e) {
  const long long m = (long long)((int32_t)e >> 31);  // 0 or -1
  return (v ^ m) - m;
}

// ------------------------------------------------------------------ start vectors
__device__ __forceinline__ long long shift_signed(long long v, int sh) {
  if (sh >= 0) return v << sh;
  return round_shift((i128)v, sh);
}

// X_i = (2 u_i - 1) 2^53 exactly (u_i from SplitMix64 as in ed_start_vector), moved to the
// 2^vb range.
__global__ void __launch_bounds__(kFxThreads)
fx_start_kernel(uint64_t seed, int64_t n, int64_t cols, int64_t ld, const int32_t* __restrict__ colpos,
                int vb, long long* __restrict__ X, long long* __restrict__ part) {
  I192 acc;
  i192_zero(acc);
  long long mx = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + ((uint64_t)i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    long long v = (long long)(2ull * (z >> 11)) - (1LL << 53);
    v = shift_signed(v, vb - 53);
    const int64_t r = i / cols, c = i - r * cols;
    X[r * ld + (colpos ? colpos[c] : c)] = v;
    i192_add(acc, (i128)v * v);
    mx = max(mx, v < 0 ? -v : v);
  }
  fx_block_reduce(acc, mx, part + 4 * blockIdx.x);
}

// Largest |f_i| as its IEEE bit pattern (sign cleared); a non-finite entry gives the
// pattern of infinity or NaN, which the host rejects.
__global__ void __launch_bounds__(kFxThreads)
fx_absmax_kernel(const double* __restrict__ f, int64_t n, unsigned long long* __restrict__ part) {
  __shared__ unsigned long long sm[32];
  unsigned long long m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)__double_as_longlong(f[i]) & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) part[blockIdx.x] = m;
  }
}

__global__ void fx_absmax_final(const unsigned long long* __restrict__ part, int n,
                                unsigned long long* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    unsigned long long m = 0;
    for (int i = 0; i < n; ++i) m = max(m, part[i]);
    *out = m;
  }
}

// X_i = f_i 2^(vb - E) with |f| < 2^E, by integer manipulation of the IEEE fields (round
// half up where bits fall off).
__global__ void __launch_bounds__(kFxThreads)
fx_copy_in_kernel(const double* __restrict__ f, int64_t n, int64_t cols, int64_t ld,
                  const int32_t* __restrict__ colpos, int vb, int E, long long* __restrict__ X,
                  long long* __restrict__ part) {
  I192 acc;
  i192_zero(acc);
  long long mx = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(f[i]);
    const int ef = (int)((bits >> 52) & 0x7FF);
    long long mant = (long long)(bits & 0xFFFFFFFFFFFFFull);
    int e2 = -1074;
    if (ef) {
      mant |= 1LL << 52;
      e2 = ef - 1075;
    }
    long long v = shift_signed(mant, e2 + vb - E);
    if (bits >> 63) v = -v;
    const int64_t r = i / cols, c = i - r * cols;
    X[r * ld + (colpos ? colpos[c] : c)] = v;
    i192_add(acc, (i128)v * v);
    mx = max(mx, v < 0 ? -v : v);
  }
  fx_block_reduce(acc, mx, part + 4 * blockIdx.x);
}

// f_1 = X / ||X||: scale[0] = 1 / sqrt(sum X^2), fx_max[0] = max |X|.
__global__ void __launch_bounds__(kFxThreads)
fx_init_kernel(LzScalars* S, const long long* __restrict__ part, int n) {
  I192 sum;
  long long mx;
  fx_sum_partials(part, n, sum, mx);
  if (threadIdx.x == 0) {
    const double q2 = i192_to_double(sum);
    S->scale[0] = q2 > 0.0 ? 1.0 / sqrt(q2) : 0.0;
    S->scale[1] = 0.0;
    S->fx_max[0] = mx;
    S->fx_max[1] = 0;
  }
}

// ------------------------------------------------------------------ one step
__global__ void fx_plan_kernel(LzScalars* S, int cur, double t, double U, int hops, int nmax,
                               int vb) {
  if (threadIdx.x != 0 || S->status != 0) return;
  const int j = S->j + 1;
  const double sc = S->scale[cur], sp = S->scale[1 - cur];
  const double mc = (double)S->fx_max[cur], mp = (double)S->fx_max[1 - cur];
  const double cp = sc != 0.0 ? S->beta[j] * sp / sc : 0.0;
  const double bound = (fabs(t) * hops + fabs(U) * nmax) * mc + fabs(cp) * mp;
  int r = 0;
  if (bound > 0.0 && isfinite(bound)) r = ilogb(bound) + 1 - (vb - 1);
  const double A = ldexp(-t, -r), B = ldexp(U, -r), C = ldexp(-cp, -r);
  const double M = fmax(fabs(A), fmax(fabs(B), fabs(C)));
  int k = 0;
  long long a = 0, b = 0, c = 0;
  if (M > 0.0 && isfinite(M)) {
    k = ilogb(M) - 61;
    a = llrint(ldexp(A, -k));
    b = llrint(ldexp(B, -k));
    c = llrint(ldexp(C, -k));
  }
  S->fx_a = a;
  S->fx_b = b;
  S->fx_c = c;
  S->fx_k = k;
  S->fx_r = r;
  S->fx_sw = ldexp(sc, r);
}

struct FxHvArgs {
  const uint32_t* __restrict__ up_bits;
  const uint32_t* __restrict__ dn_bits;
  const int32_t* __restrict__ hop_up;
  const int32_t* __restrict__ hop_dn;
  int64_t dim_up, dim_dn, ld;
  int maxhops_up, maxhops_dn;
};

// s += the signed values of a state's hop targets (integers: the order does not matter),
// four hops at a time with their table entries and values loaded before any is added, so a
// thread has more loads in flight. tab[k * stride] is hop k's entry; a target >= n is
// padding, and the rest of the state's list is padding too.
template <typename Load>
__device__ __forceinline__ void fx_add_hops(long long& s, const int32_t* tab, int64_t stride, int mh,
                                            int64_t n, Load load) {
  int k = 0;
  for (; k + 4 <= mh; k += 4) {
    uint32_t e[4];
    long long v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) e[q] = (uint32_t)tab[(int64_t)(k + q) * stride];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t tg = (int64_t)(e[q] & kTargetMask);
      v[q] = tg < n ? sgn_apply(load(tg), e[q]) : 0LL;
    }
    s += (v[0] + v[1]) + (v[2] + v[3]);
    if ((int64_t)(e[3] & kTargetMask) >= n) return;
  }
  for (; k < mh; ++k) {
    const uint32_t e = (uint32_t)tab[(int64_t)k * stride];
    const int64_t tg = (int64_t)(e & kTargetMask);
    if (tg >= n) return;
    s += sgn_apply(load(tg), e);
  }
}

// W = round((a S + b n X + c P) 2^k), written over P; partial sums of W X (exact).
// Row-staged like hv_staged_kernel: R up rows per CTA, interleaved in shared memory.
template <int R>
__global__ void __launch_bounds__(kFxThreads)
fx_hv_staged_kernel(FxHvArgs a, const long long* __restrict__ x, long long* __restrict__ y,
                    const LzScalars* __restrict__ S, long long* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (S->status != 0) return;
  const long long ca = S->fx_a, cb = S->fx_b, cc = S->fx_c;
  const int k = S->fx_k;
  const int dn = (int)a.dim_dn;
  long long* xs = reinterpret_cast<long long*>(smem);
  int32_t* ut = reinterpret_cast<int32_t*>(xs + (size_t)(dn + 1) * R);
  const int64_t u0 = (int64_t)blockIdx.x * R;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t u = u0 + r;
    const long long* xr = x + u * a.ld;
    for (int d = threadIdx.x; d < dn; d += blockDim.x) xs[d * R + r] = (u < a.dim_up) ? xr[d] : 0LL;
  }
  if (threadIdx.x < R) xs[(size_t)dn * R + threadIdx.x] = 0LL;
  for (int i = threadIdx.x; i < R * a.maxhops_up; i += blockDim.x) {
    const int r = i / a.maxhops_up, kk = i - r * a.maxhops_up;
    const int64_t u = u0 + r;
    ut[i] = (u < a.dim_up) ? a.hop_up[(int64_t)kk * a.dim_up + u] : (int32_t)a.dim_up;
  }
  uint32_t ub[R];
#pragma unroll
  for (int r = 0; r < R; ++r) ub[r] = (u0 + r < a.dim_up) ? a.up_bits[u0 + r] : 0u;
  __syncthreads();

  I192 dot;
  i192_zero(dot);
  for (int d = threadIdx.x; d < dn; d += blockDim.x) {
    const uint32_t db = a.dn_bits[d];
    long long hs[R];
#pragma unroll
    for (int r = 0; r < R; ++r) hs[r] = 0;
    for (int kk = 0; kk < a.maxhops_dn; ++kk) {
      const uint32_t e = (uint32_t)a.hop_dn[(int64_t)kk * dn + d];
      const int tg = (int)(e & kTargetMask);
#pragma unroll
      for (int r = 0; r < R; ++r) hs[r] += sgn_apply(xs[tg * R + r], e);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t u = u0 + r;
      if (u < a.dim_up) {
        fx_add_hops(hs[r], ut + r * a.maxhops_up, 1, a.maxhops_up, a.dim_up,
                    [&](int64_t tg) { return x[tg * a.ld + d]; });
        const long long xc = xs[d * R + r];
        const long long nx = xc * (long long)__popc(ub[r] & db);
        long long* yp = y + u * a.ld + d;
        const i128 p = (i128)ca * hs[r] + (i128)cb * nx + (i128)cc * (*yp);
        const long long w = round_shift(p, k);
        *yp = w;
        i192_add(dot, (i128)w * xc);
      }
    }
  }
  fx_block_reduce(dot, 0, part + 4 * blockIdx.x);
}

// Fallback when a row does not fit in shared memory.
__global__ void __launch_bounds__(kFxThreads)
fx_hv_global_kernel(FxHvArgs a, const long long* __restrict__ x, long long* __restrict__ y,
                    const LzScalars* __restrict__ S, long long* __restrict__ part) {
  if (S->status != 0) return;
  const long long ca = S->fx_a, cb = S->fx_b, cc = S->fx_c;
  const int k = S->fx_k;
  I192 dot;
  i192_zero(dot);
  const int64_t total = a.dim_up * a.dim_dn;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = g / a.dim_dn, d = g - u * a.dim_dn;
    const long long* xr = x + u * a.ld;
    long long hs = 0;
    fx_add_hops(hs, a.hop_dn + d, a.dim_dn, a.maxhops_dn, a.dim_dn, [&](int64_t tg) { return xr[tg]; });
    fx_add_hops(hs, a.hop_up + u, a.dim_up, a.maxhops_up, a.dim_up,
                [&](int64_t tg) { return x[tg * a.ld + d]; });
    const long long xc = xr[d];
    const long long nx = xc * (long long)__popc(a.up_bits[u] & a.dn_bits[d]);
    long long* yp = y + u * a.ld + d;
    const long long w = round_shift((i128)ca * hs + (i128)cb * nx + (i128)cc * (*yp), k);
    *yp = w;
    i192_add(dot, (i128)w * xc);
  }
  fx_block_reduce(dot, 0, part + 4 * blockIdx.x);
}

__global__ void __launch_bounds__(kFxThreads)
fx_update_kernel(LzScalars* S, int cur, const long long* __restrict__ xc, long long* __restrict__ xp,
                 int64_t n, const long long* __restrict__ pa, int na, long long* __restrict__ pb) {
  if (S->status != 0) return;
  I192 sum;
  long long unused;
  fx_sum_partials(pa, na, sum, unused);
  const double sc = S->scale[cur], sw = S->fx_sw;
  const double alpha = sw * sc * i192_to_double(sum);
  if (blockIdx.x == 0 && threadIdx.x == 0) S->alpha[S->j + 1] = alpha;
  const double D = -alpha * (sc / sw);
  long long d = 0;
  int k2 = -1;
  if (D != 0.0 && isfinite(D)) {
    k2 = ilogb(D) - 61;
    d = llrint(ldexp(D, -k2));
  }
  A192 q2;
  long long mx = 0;
  // n is even (rows are padded to 32 elements): pairs of elements, two pairs in flight
  const longlong2* c2 = reinterpret_cast<const longlong2*>(xc);
  longlong2* p2 = reinterpret_cast<longlong2*>(xp);
  const int64_t n2 = n / 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  auto upd = [&](long long w, long long c) {
    const long long q = w + round_shift128(smul128(d, c), k2);
    const unsigned long long aq = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
    a192_add_sq(q2, aq);
    mx = max(mx, (long long)aq);
    return q;
  };
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += 2 * stride) {
    const bool two = i + stride < n2;
    const longlong2 w0 = p2[i], c0 = c2[i];
    longlong2 w1 = make_longlong2(0, 0), c1 = make_longlong2(0, 0);
    if (two) {
      w1 = p2[i + stride];
      c1 = c2[i + stride];
    }
    p2[i] = make_longlong2(upd(w0.x, c0.x), upd(w0.y, c0.y));
    if (two) p2[i + stride] = make_longlong2(upd(w1.x, c1.x), upd(w1.y, c1.y));
  }
  fx_block_reduce(a192_get(q2), mx, pb + 4 * blockIdx.x);
}

__global__ void __launch_bounds__(kRedThreads)
fx_finish_kernel(LzScalars* S, int cur, const long long* __restrict__ pb, int nb) {
  __shared__ int stop_s;
  if (S->status != 0) return;
  const int j = S->j + 1;
  I192 sum;
  long long mx;
  fx_sum_partials(pb, nb, sum, mx);
  if (threadIdx.x == 0) {
    const double sw = S->fx_sw;
    const double beta = sw * sqrt(i192_to_double(sum));
    stop_s = finish_record_beta(S, j, beta);
    if (stop_s == 0) {
      S->scale[1 - cur] = sw / beta;
      S->fx_max[1 - cur] = mx;
    }
  }
  __syncthreads();
  finish_tail(S, j, stop_s);
}

// ------------------------------------------------------------------ ground-state vector
// psi = sum_j y_j f_j accumulated in int64 with psi = 2^-60 P (|psi_i| stays below 4):
// P_i += round(c X_i 2^k) with c 2^k = y_j s_cur 2^60. Also tracks the index of the
// largest |P| (ties: lowest index) for the sign gauge.
__global__ void __launch_bounds__(kFxThreads)
fx_psi_accum_kernel(const LzScalars* __restrict__ S, int cur, const double* __restrict__ y, int jstep,
                    const long long* __restrict__ X, int64_t rows, int64_t cols, int64_t ld,
                    const int32_t* __restrict__ colpos, long long* __restrict__ P) {
  const double c = y[jstep] * S->scale[cur] * 0x1.0p60;
  long long m = 0;
  int k = -1;
  if (c != 0.0 && isfinite(c)) {
    k = ilogb(c) - 61;
    m = llrint(ldexp(c, -k));
  }
  const int64_t n = rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / cols, cc = i - r * cols;
    P[i] += round_shift((i128)m * X[r * ld + (colpos ? colpos[cc] : cc)], k);
  }
}

// Largest |P_i| and its lowest index: partial records (value, index) per CTA.
__global__ void __launch_bounds__(kFxThreads)
fx_psi_argmax_kernel(const long long* __restrict__ P, int64_t n, long long* __restrict__ part) {
  __shared__ long long sv[kFxThreads];
  __shared__ long long si[kFxThreads];
  long long bv = -1, bi = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const long long v = P[i] < 0 ? -P[i] : P[i];
    if (v > bv) {
      bv = v;
      bi = i;
    }
  }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const long long v2 = sv[threadIdx.x + o], i2 = si[threadIdx.x + o];
      if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sv[0];
    part[2 * blockIdx.x + 1] = si[0];
  }
}

// psi (FP64) = gauge * P 2^-60 / ||P 2^-60||, gauge making the largest entry positive.
__global__ void __launch_bounds__(kFxThreads)
fx_psi_out_kernel(const long long* __restrict__ P, int64_t n, const long long* __restrict__ amax,
                  int namax, const long long* __restrict__ nrm_part, int nn, double* __restrict__ out) {
  __shared__ long long best_i;
  if (threadIdx.x == 0) {
    long long bv = -1, bi = 0;
    for (int b = 0; b < namax; ++b) {
      const long long v = amax[2 * b], i = amax[2 * b + 1];
      if (v > bv || (v == bv && i < bi)) {
        bv = v;
        bi = i;
      }
    }
    best_i = bi;
  }
  I192 sum;
  long long unused;
  fx_sum_partials(nrm_part, nn, sum, unused);
  const double nrm = sqrt(i192_to_double(sum));
  const double g = (P[best_i] < 0 ? -1.0 : 1.0) / nrm;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)P[i] * g;
}

// Partial sums of P_i^2 (exact).
__global__ void __launch_bounds__(kFxThreads)
fx_psi_norm_kernel(const long long* __restrict__ P, int64_t n, long long* __restrict__ part) {
  I192 acc;
  i192_zero(acc);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    i192_add(acc, (i128)P[i] * P[i]);
  fx_block_reduce(acc, 0, part + 4 * blockIdx.x);
}

// ------------------------------------------------------------------ host side
static int fx_red_grid(int64_t n) {
  const int64_t want = (n + kFxThreads - 1) / kFxThreads;
  const int64_t cap = (int64_t)sm_count() * 4;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

static FxHvArgs fx_args(const ed_basis* b, int64_t ld) {
  FxHvArgs a;
  a.up_bits = b->up.bits;
  a.dn_bits = b->dn.bits;
  a.hop_up = b->up.hop;
  a.hop_dn = b->dn.hop;
  a.dim_up = b->up.dim;
  a.dim_dn = b->dn.dim;
  a.ld = ld;
  a.maxhops_up = b->up.maxhops;
  a.maxhops_dn = b->dn.maxhops;
  return a;
}

template <int R>
static size_t fx_smem(const ed_basis* b) {
  return (size_t)(b->dn.dim + 1) * R * 8 + (size_t)R * b->up.maxhops * 4;
}

static int smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

static int fx_rows(const ed_basis* b) {
  if (b->up.dim < kMinRowsStaged) return 0;  // few rows: the element-parallel kernel
  const size_t lim = (size_t)smem_optin();
  if (fx_smem<2>(b) <= lim && b->up.dim >= 2) return 2;
  if (fx_smem<1>(b) <= lim) return 1;
  return 0;
}

ed_status fx_psi_accum(const ed_basis* b, const LzScalars* S, int cur, const double* y, int j,
                       const long long* X, int64_t ld, const int32_t* colpos, long long* P,
                       cudaStream_t s) {
  fx_psi_accum_kernel<<<fx_red_grid(b->dim), kFxThreads, 0, s>>>(S, cur, y, j, X, b->up.dim,
                                                                  b->dn.dim, ld, colpos, P);
  ED_TRY_CUDA(cudaGetLastError());
  return ED_OK;
}

ed_status fx_psi_finish(const ed_basis* b, const long long* P, long long* part, double* out,
                        cudaStream_t s) {
  const int g = fx_red_grid(b->dim);
  fx_psi_argmax_kernel<<<g, kFxThreads, 0, s>>>(P, b->dim, part);
  fx_psi_norm_kernel<<<g, kFxThreads, 0, s>>>(P, b->dim, part + 2 * g);
  fx_psi_out_kernel<<<g, kFxThreads, 0, s>>>(P, b->dim, part, g, part + 2 * g, g, out);
  ED_TRY_CUDA(cudaGetLastError());
  return ED_OK;
}

ed_status fx_prepare(const ed_basis* b) {
  const int R = fx_rows(b);
  if (R == 2)
    ED_TRY_CUDA(allow_max_smem(fx_hv_staged_kernel<2>));
  if (R == 1)
    ED_TRY_CUDA(allow_max_smem(fx_hv_staged_kernel<1>));
  return ED_OK;
}

ed_status fx_start(const ed_basis* b, const FxRun& fx, uint64_t seed, long long* X, int64_t ld,
                   const int32_t* colpos, LzScalars* S, long long* part, cudaStream_t s) {
  const int g = fx_red_grid(b->dim);
  fx_start_kernel<<<g, kFxThreads, 0, s>>>(seed, b->dim, b->dn.dim, ld, colpos, fx.vb, X, part);
  fx_init_kernel<<<1, kFxThreads, 0, s>>>(S, part, g);
  ED_TRY_CUDA(cudaGetLastError());
  return ED_OK;
}

ed_status fx_copy_in(const ed_basis* b, const FxRun& fx, const double* f1, long long* X,
                     int64_t ld, const int32_t* colpos, LzScalars* S, long long* part,
                     cudaStream_t s) {
  const int g = fx_red_grid(b->dim);
  unsigned long long* pm = reinterpret_cast<unsigned long long*>(part);
  fx_absmax_kernel<<<g, kFxThreads, 0, s>>>(f1, b->dim, pm);
  fx_absmax_final<<<1, 32, 0, s>>>(pm, g, pm + g);
  ED_TRY_CUDA(cudaGetLastError());
  unsigned long long mb = 0;
  ED_TRY_CUDA(cudaMemcpyAsync(&mb, pm + g, sizeof(mb), cudaMemcpyDeviceToHost, s));
  ED_TRY_CUDA(cudaStreamSynchronize(s));
  const int ef = (int)(mb >> 52);
  ED_CHECK_ARG(ef != 0x7FF, "f1 holds a non-finite value");
  ED_CHECK_ARG(mb != 0, "f1 is the zero vector");
  const int E = ef ? ef - 1022 : -1022;  // |f1| < 2^E
  fx_copy_in_kernel<<<g, kFxThreads, 0, s>>>(f1, b->dim, b->dn.dim, ld, colpos, fx.vb, E, X,
                                              part);
  fx_init_kernel<<<1, kFxThreads, 0, s>>>(S, part, g);
  ED_TRY_CUDA(cudaGetLastError());
  return ED_OK;
}

ed_status fx_step(const ed_basis* b, const FxRun& fx, double t, double U, long long* const B[2],
                  int cur, int64_t ld, LzScalars* S, long long* pa, long long* pb,
                  cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, const Hv2Plan* plan,
                  const Reorth* ro) {
  fx_plan_kernel<<<1, 32, 0, s>>>(S, cur, t, U, fx.hops, fx.nmax, fx.vb);
  if (ev0) ED_TRY_CUDA(cudaEventRecord(ev0, s));
  const FxHvArgs a = fx_args(b, ld);
  const int R = plan ? -1 : fx_rows(b);
  int grid;
  if (plan) {
    grid = hv2_grid(plan);
    ed_status r = hv2_launch(plan, b, t, U, B[cur], B[1 - cur], S, cur, pa, s);
    if (r != ED_OK) return r;
  } else if (R == 2) {
    grid = (int)((b->up.dim + 1) / 2);
    fx_hv_staged_kernel<2><<<grid, kFxThreads, fx_smem<2>(b), s>>>(a, B[cur], B[1 - cur], S, pa);
  } else if (R == 1) {
    grid = (int)b->up.dim;
    fx_hv_staged_kernel<1><<<grid, kFxThreads, fx_smem<1>(b), s>>>(a, B[cur], B[1 - cur], S, pa);
  } else {
    grid = fx_red_grid(b->dim) * 2;
    fx_hv_global_kernel<<<grid, kFxThreads, 0, s>>>(a, B[cur], B[1 - cur], S, pa);
  }
  ED_TRY_CUDA(cudaGetLastError());
  if (ev1) ED_TRY_CUDA(cudaEventRecord(ev1, s));
  const int64_t n = b->up.dim * ld;
  const int ug = fx_red_grid(n);
  fx_update_kernel<<<ug, kFxThreads, 0, s>>>(S, cur, B[cur], B[1 - cur], n, pa, grid, pb);
  if (ro) {
    const ed_status r = ro_apply(ro, S, B[1 - cur], pb, ug, s);
    if (r != ED_OK) return r;
  }
  fx_finish_kernel<<<1, kRedThreads, 0, s>>>(S, cur, pb, ug);
  ED_TRY_CUDA(cudaGetLastError());
  if (ro) return ro_store(ro, S, 1 - cur, B[1 - cur], s);
  return ED_OK;
}

}  // namespace ed

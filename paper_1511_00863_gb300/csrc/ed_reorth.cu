// Reorthogonalisation of the Lanczos residual on the device (ed_opts.reorth = 1 full,
// 2 partial).
//
// Algorithm 1 (Sec. 2.2) as printed keeps only the last two vectors; in finite precision the
// vectors lose orthogonality once a Ritz value converges, and copies ("ghosts") of converged
// eigenvalues appear in T_m. With a reorthogonalisation mode the run also keeps every
// Lanczos vector f_1 .. f_j in device memory (same storage as the run: FP32, FP64, or int64
// fixed point with one FP64 scale per vector) and, after q = w - a_j f_j, removes from q its
// components along the stored vectors by classical Gram-Schmidt, two passes:
//     h_i = f_i . q   (i = 1..j),   q -= sum_i h_i f_i.
// In the buffers' own units (f_i = s_i V_i, q = s_q Q) a pass is Q -= sum_i s_i^2 (V_i . Q) V_i.
// The dot products are accumulated in FP64 (FP64 runs), as compensated FP32 pairs summed in
// FP64 per CTA (FP32 runs), or exactly in 192-bit integers (fixed-point runs); the
// fixed-point correction sum_i c_i V_i is formed exactly from 64-bit mantissas of the
// coefficients and rounded once per element.
//
// Partial mode follows Simon's partial reorthogonalisation (H. D. Simon, Math. Comp. 42
// (1984) 115-142): the level of orthogonality omega_{j+1,k} = f_{j+1} . f_k is estimated from
// the recurrence the Lanczos relation implies,
//   b_{j+1} omega_{j+1,k} = b_{k+1} omega_{j,k+1} + (a_k - a_j) omega_{j,k} + b_k omega_{j,k-1}
//                           - b_j omega_{j-1,k}  (+ a rounding term),
// with omega_{k,k} = 1 and omega_{k+1,k} = psi (the local level); when some |omega_{j+1,k}|
// exceeds sqrt(eps) the residual is reorthogonalised against all stored vectors, at this
// step and the next, and the estimates are reset to psi.
// Every kernel returns at entry once the run has stopped (S->status != 0) or, for the
// passes, when the step does not reorthogonalise.
#include <cmath>
#include <type_traits>

#include "ed_fixed.cuh"
#include "ed_internal.cuh"
#include "ed_lanczos_dev.cuh"

namespace ed {

constexpr int kRoThreads = 256;
constexpr int kRoBatch = 8;  // stored vectors per sweep of the dot-product kernel

struct RoFlags {
  int flag;     // reorthogonalise the current step
  int pending;  // the next step must reorthogonalise too (partial mode)
  int count;    // steps reorthogonalised so far
  int pad_;
};

struct Reorth {
  int mode = 0;        // 1 full, 2 partial, 3 store only (the mixed-precision solve)
  int kind = 0;        // 0 FP32, 1 FP64, 2 int64 fixed point
  int64_t n = 0;       // elements per stored vector (padded layout)
  int slots = 0;       // stored vectors (max_steps + 1)
  int G = 0;           // CTAs of the dot-product kernel
  void* V = nullptr;   // [slots][n]
  double* vscale = nullptr;  // [slots]
  double* coef = nullptr;    // [slots]
  void* part = nullptr;      // [slots][G] doubles, or [slots][G][3] words (fixed point)
  double* omega = nullptr;   // [3][slots + 2]
  RoFlags* F = nullptr;
  double eps = 0.0, psi = 0.0;
};

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ void i192_from_words(I192& a, long long w0, long long w1, long long w2) {
  a.lo = ((u128)(unsigned long long)w1 << 64) | (u128)(unsigned long long)w0;
  a.hi = w2;
}

// round(v 2^-s) for 0 < s < 190, the result known to fit in 64 bits (round half up).
__device__ __forceinline__ long long i192_round_shift(I192 v, int s) {
  if (s <= 0) return (long long)((unsigned long long)v.lo << (-s));
  if (s <= 128) {  // add 2^(s-1) to the 192-bit value
    const u128 h = (u128)1 << (s - 1);
    const u128 lo = v.lo + h;
    v.hi += (lo < v.lo) ? 1 : 0;
    v.lo = lo;
  } else {
    v.hi += 1LL << (s - 129);
  }
  if (s >= 128) return v.hi >> (s - 128);
  if (s >= 64)
    return (long long)(unsigned long long)((v.lo >> s) | ((u128)(unsigned long long)v.hi << (128 - s)));
  return (long long)(unsigned long long)(v.lo >> s);
}

// Exact block sum of a 192-bit value; the result is valid in thread 0.
__device__ __forceinline__ I192 ro_block_sum192(I192 v, unsigned long long (*sm)[3]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const I192 w = i192_shfl_down(v, o);
    i192_add(v, w);
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) {
    sm[wid][0] = (unsigned long long)v.lo;
    sm[wid][1] = (unsigned long long)(v.lo >> 64);
    sm[wid][2] = (unsigned long long)v.hi;
  }
  __syncthreads();
  I192 a;
  i192_zero(a);
  if (wid == 0) {
    if (lane < (int)(blockDim.x >> 5))
      i192_from_words(a, (long long)sm[lane][0], (long long)sm[lane][1], (long long)sm[lane][2]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const I192 w = i192_shfl_down(a, o);
      i192_add(a, w);
    }
  }
  __syncthreads();
  return a;
}

template <typename T> struct RoAcc;
template <> struct RoAcc<float> { typedef DotAcc<float> type; };
template <> struct RoAcc<double> { typedef DotAcc<double> type; };

// ------------------------------------------------------------------ store f_{j+1}
// Slot S->j receives the buffer that holds f_{S->j + 1} (at the start of a run S->j = 0 and
// the buffer holds f_1) and its scale.
template <typename T>
__global__ void __launch_bounds__(kRoThreads)
ro_store_kernel(const LzScalars* __restrict__ S, int buf, const T* __restrict__ src,
                T* __restrict__ V, double* __restrict__ vscale, int64_t n, int slots) {
  if (S->status != 0) return;
  const int slot = S->j;
  if (slot >= slots) return;
  T* dst = V + (int64_t)slot * n;
  // n is a multiple of 32 elements: 16-byte vectors
  const int4* s4 = reinterpret_cast<const int4*>(src);
  int4* d4 = reinterpret_cast<int4*>(dst);
  const int64_t nv = n * (int64_t)sizeof(T) / 16;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv;
       i += (int64_t)gridDim.x * blockDim.x)
    d4[i] = s4[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) vscale[slot] = S->scale[buf];
}

// ------------------------------------------------------------------ decide (one CTA)
// ||q||^2 from the update pass's partials: FP64 partial sums, or (fixed point) exact records
// (lo, lo >> 64, hi, max) scaled by s_w^2.
__device__ __forceinline__ double ro_q_norm2(const LzScalars* S, const void* pb, int nb, int kind,
                                             double* red, unsigned long long (*sm)[3]) {
  __shared__ double out;
  if (kind != 2) {
    const double v = block_sum_array(reinterpret_cast<const double*>(pb), nb, red);
    return v;
  }
  const long long* p = reinterpret_cast<const long long*>(pb);
  I192 acc;
  i192_zero(acc);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    I192 w;
    i192_from_words(w, p[4 * i], p[4 * i + 1], p[4 * i + 2]);
    i192_add(acc, w);
  }
  const I192 tot = ro_block_sum192(acc, sm);
  if (threadIdx.x == 0) out = i192_to_double(tot) * S->fx_sw * S->fx_sw;
  __syncthreads();
  return out;
}

__global__ void __launch_bounds__(kRoThreads)
ro_decide_kernel(const LzScalars* __restrict__ S, RoFlags* __restrict__ F, double* __restrict__ omega,
                 int mode, int kind, const void* __restrict__ pb, int nb, int slots, double eps,
                 double psi) {
  __shared__ double red[33];
  __shared__ unsigned long long sm[32][3];
  __shared__ float mx_s;
  if (S->status != 0) return;
  const int j = S->j + 1;
  if (mode == 1) {
    if (threadIdx.x == 0) {
      F->flag = 1;
      F->count += 1;
    }
    return;
  }
  const double bq = sqrt(ro_q_norm2(S, pb, nb, kind, red, sm));  // b_{j+1} before the passes
  const int W = slots + 2;
  double* om_prev = omega + (size_t)((j + 2) % 3) * W;  // omega_{j-1, k}
  double* om_cur = omega + (size_t)(j % 3) * W;         // omega_{j, k}
  double* om_new = omega + (size_t)((j + 1) % 3) * W;   // omega_{j+1, k}
  if (threadIdx.x == 0) mx_s = 0.f;
  __syncthreads();
  const double* a = S->alpha;
  const double* b = S->beta;  // b[1] = 0
  float mx = 0.f;
  for (int k = 1 + threadIdx.x; k <= j - 1; k += blockDim.x) {
    double v = b[k + 1] * om_cur[k + 1] + (a[k] - a[j]) * om_cur[k] +
               (k > 1 ? b[k] * om_cur[k - 1] : 0.0) - b[j] * om_prev[k];
    const double th = psi * (b[k + 1] + bq);  // rounding term, taken with the sign of v
    v = (v + (v >= 0.0 ? th : -th)) / bq;
    om_new[k] = v;
    mx = fmaxf(mx, (float)fabs(v));
  }
  if (mx > 0.f) atomicMax(reinterpret_cast<int*>(&mx_s), __float_as_int(mx));  // mx >= 0
  __syncthreads();
  const bool est = (double)mx_s > sqrt(eps);
  const bool flag = est || F->pending != 0;
  if (flag)
    for (int k = 1 + threadIdx.x; k <= j - 1; k += blockDim.x) om_new[k] = psi;
  if (threadIdx.x == 0) {
    om_new[0] = 0.0;
    om_new[j] = psi;
    om_new[j + 1] = 1.0;
    F->flag = flag ? 1 : 0;
    F->pending = (est && F->pending == 0) ? 1 : 0;
    if (flag) F->count += 1;
  }
}

// ------------------------------------------------------------------ pass: dot products
// part[i * G + cta] = partial of V_i . Q over the CTA's element range (fixed point: exact
// 192-bit records of 3 words at [(i * G + cta) * 3]).
template <typename T>
__global__ void __launch_bounds__(kRoThreads)
ro_dots_kernel(const LzScalars* __restrict__ S, const RoFlags* __restrict__ F,
               const T* __restrict__ Q, const T* __restrict__ V, int64_t n, void* __restrict__ part) {
  __shared__ double red[33];
  __shared__ unsigned long long sm[32][3];
  if (S->status != 0 || F->flag == 0) return;
  const int j = S->j + 1;  // f_1 .. f_j in slots 0 .. j-1
  const int G = gridDim.x;
  const int64_t chunk = (n + G - 1) / G;
  const int64_t e0 = (int64_t)blockIdx.x * chunk;
  const int64_t e1 = e0 + chunk < n ? e0 + chunk : n;
  for (int i0 = 0; i0 < j; i0 += kRoBatch) {
    if constexpr (sizeof(T) == 8 && !std::is_floating_point<T>::value) {
      A192 acc[kRoBatch];
      for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const long long q = (long long)Q[e];
#pragma unroll
        for (int r = 0; r < kRoBatch; ++r)
          if (i0 + r < j) a192_add_prod(acc[r], (long long)V[(int64_t)(i0 + r) * n + e], q);
      }
#pragma unroll
      for (int r = 0; r < kRoBatch; ++r) {
        if (i0 + r >= j) break;
        const I192 tot = ro_block_sum192(a192_get(acc[r]), sm);
        if (threadIdx.x == 0) {
          long long* o = reinterpret_cast<long long*>(part) + ((int64_t)(i0 + r) * G + blockIdx.x) * 3;
          o[0] = (long long)(unsigned long long)tot.lo;
          o[1] = (long long)(unsigned long long)(tot.lo >> 64);
          o[2] = tot.hi;
        }
      }
    } else {
      typename RoAcc<T>::type acc[kRoBatch];
      for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const T q = Q[e];
#pragma unroll
        for (int r = 0; r < kRoBatch; ++r)
          if (i0 + r < j) acc[r].add(V[(int64_t)(i0 + r) * n + e], q);
      }
#pragma unroll
      for (int r = 0; r < kRoBatch; ++r) {
        if (i0 + r >= j) break;
        const double v = block_sum(acc[r].get(), red);
        if (threadIdx.x == 0) reinterpret_cast<double*>(part)[(int64_t)(i0 + r) * G + blockIdx.x] = v;
      }
    }
  }
}

// coef[i] = s_i^2 (V_i . Q), one CTA per stored vector (CTAs past j return).
__global__ void __launch_bounds__(kRoThreads)
ro_coef_kernel(const LzScalars* __restrict__ S, const RoFlags* __restrict__ F, int kind,
               const void* __restrict__ part, int G, const double* __restrict__ vscale,
               double* __restrict__ coef) {
  __shared__ double red[33];
  __shared__ unsigned long long sm[32][3];
  if (S->status != 0 || F->flag == 0) return;
  const int j = S->j + 1;
  const int i = blockIdx.x;
  if (i >= j) return;
  double d;
  if (kind != 2) {
    d = block_sum_array(reinterpret_cast<const double*>(part) + (int64_t)i * G, G, red);
  } else {
    const long long* p = reinterpret_cast<const long long*>(part) + (int64_t)i * G * 3;
    I192 acc;
    i192_zero(acc);
    for (int c = threadIdx.x; c < G; c += blockDim.x) {
      I192 w;
      i192_from_words(w, p[3 * c], p[3 * c + 1], p[3 * c + 2]);
      i192_add(acc, w);
    }
    const I192 tot = ro_block_sum192(acc, sm);
    d = i192_to_double(tot);  // valid in thread 0
  }
  if (threadIdx.x == 0) coef[i] = vscale[i] * vscale[i] * d;
}

// ------------------------------------------------------------------ pass: update
// Q -= sum_i coef[i] V_i; on the last pass also the partial records of ||Q||^2 (and max |Q|
// for fixed point) in the update pass's format, so the finish kernel reads them unchanged.
template <typename T>
__global__ void __launch_bounds__(kRoThreads)
ro_update_kernel(const LzScalars* __restrict__ S, const RoFlags* __restrict__ F,
                 T* __restrict__ Q, const T* __restrict__ V, int64_t n,
                 const double* __restrict__ coef, int last, void* __restrict__ pb) {
  extern __shared__ __align__(16) unsigned char ro_smem[];
  __shared__ double red[33];
  __shared__ int K_s;
  __shared__ unsigned mxe_s;
  if (S->status != 0 || F->flag == 0) return;
  const int j = S->j + 1;
  if constexpr (sizeof(T) == 8 && !std::is_floating_point<T>::value) {
    // common exponent K: coef[i] = m_i 2^K with |m_i| < 2^62 for the largest coefficient
    long long* m = reinterpret_cast<long long*>(ro_smem);
    if (threadIdx.x == 0) mxe_s = 0u;
    __syncthreads();
    unsigned me = 0u;
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
      const double c = coef[i];
      if (c != 0.0 && isfinite(c)) me = max(me, (unsigned)(ilogb(c) + 2048));
    }
    atomicMax(&mxe_s, me);
    __syncthreads();
    if (threadIdx.x == 0) K_s = mxe_s ? (int)mxe_s - 2048 - 61 : 0;
    __syncthreads();
    const int K = K_s;
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
      const double c = coef[i];
      m[i] = (mxe_s && isfinite(c)) ? llrint(ldexp(c, -K)) : 0LL;
    }
    __syncthreads();
    A192 q2;
    long long mx = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
      A192 acc;
      for (int i = 0; i < j; ++i) a192_add_prod(acc, m[i], (long long)V[(int64_t)i * n + e]);
      const long long corr = mxe_s ? i192_round_shift(a192_get(acc), -K) : 0LL;
      const long long q = (long long)Q[e] - corr;
      Q[e] = (T)q;
      if (last) {
        const unsigned long long aq = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
        a192_add_sq(q2, aq);
        mx = max(mx, (long long)aq);
      }
    }
    if (last) {
      __shared__ unsigned long long sm[32][3];
      const I192 tot = ro_block_sum192(a192_get(q2), sm);
      // max |Q| over the block
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, (long long)__shfl_down_sync(0xffffffffu, mx, o));
      __shared__ long long mxw[32];
      if ((threadIdx.x & 31) == 0) mxw[threadIdx.x >> 5] = mx;
      __syncthreads();
      if (threadIdx.x == 0) {
        long long M = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) M = max(M, mxw[w]);
        long long* o = reinterpret_cast<long long*>(pb) + 4 * blockIdx.x;
        o[0] = (long long)(unsigned long long)tot.lo;
        o[1] = (long long)(unsigned long long)(tot.lo >> 64);
        o[2] = tot.hi;
        o[3] = M;
      }
    }
  } else {
    T* c = reinterpret_cast<T*>(ro_smem);
    for (int i = threadIdx.x; i < j; i += blockDim.x) c[i] = (T)coef[i];
    __syncthreads();
    DotAcc<T> q2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
      T corr = T(0);
      for (int i = 0; i < j; ++i) corr = fma(c[i], V[(int64_t)i * n + e], corr);
      const T q = Q[e] - corr;
      Q[e] = q;
      if (last) q2.add(q, q);
    }
    if (last) {
      const double v = block_sum(q2.get(), red);
      if (threadIdx.x == 0) reinterpret_cast<double*>(pb)[blockIdx.x] = v;
    }
  }
}

// ------------------------------------------------------------------ host side
static int ro_kind(ed_dtype d) { return d == ED_F32 ? 0 : d == ED_F64 ? 2 : 1; }
static size_t ro_esize(int kind) { return kind == 0 ? 4 : 8; }

void ro_free(Reorth* r) {
  if (!r) return;
  if (r->V) cudaFree(r->V);
  if (r->vscale) cudaFree(r->vscale);
  if (r->coef) cudaFree(r->coef);
  if (r->part) cudaFree(r->part);
  if (r->omega) cudaFree(r->omega);
  if (r->F) cudaFree(r->F);
  delete r;
}

ed_status ro_create(int mode, ed_dtype dtype, int64_t n, int max_steps, int64_t dim,
                    Reorth** out) {
  *out = nullptr;
  Reorth* r = new Reorth();
  r->mode = mode;
  r->kind = ro_kind(dtype);
  r->n = n;
  r->slots = max_steps + 1;
  r->G = 2 * sm_count();
  r->eps = r->kind == 0 ? 0x1.0p-24 : 0x1.0p-53;
  // local level of orthogonality of consecutive vectors (rounding of one dot product of dim
  // terms, random-walk growth)
  r->psi = r->eps * 0.5 * sqrt((double)(dim > 1 ? dim : 1));
  const size_t vbytes = (size_t)r->slots * (size_t)n * ro_esize(r->kind);
  if (cudaMalloc(&r->V, vbytes) != cudaSuccess) {
    cudaGetLastError();
    ro_free(r);
    set_error("reorthogonalisation: out of device memory for %d stored vectors (%.2f GB); "
              "lower max_steps", max_steps + 1, (double)vbytes / 1e9);
    return ED_ERR_OOM;
  }
  const size_t pw = r->kind == 2 ? 3 : 1;
  if (cudaMalloc((void**)&r->vscale, (size_t)r->slots * 8) != cudaSuccess ||
      cudaMalloc((void**)&r->coef, (size_t)r->slots * 8) != cudaSuccess ||
      cudaMalloc(&r->part, (size_t)r->slots * r->G * pw * 8) != cudaSuccess ||
      cudaMalloc((void**)&r->omega, (size_t)3 * (r->slots + 2) * 8) != cudaSuccess ||
      cudaMalloc((void**)&r->F, sizeof(RoFlags)) != cudaSuccess) {
    cudaGetLastError();
    ro_free(r);
    set_error("reorthogonalisation: out of device memory");
    return ED_ERR_OOM;
  }
  *out = r;
  return ED_OK;
}

template <typename T>
static void ro_store_t(const Reorth* r, const LzScalars* S, int buf, const void* src, cudaStream_t s) {
  const int64_t nv = r->n * (int64_t)sizeof(T) / 16;
  int g = (int)((nv + kRoThreads - 1) / kRoThreads);
  const int cap = 4 * sm_count();
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  ro_store_kernel<T><<<g, kRoThreads, 0, s>>>(S, buf, (const T*)src, (T*)r->V, r->vscale, r->n,
                                              r->slots);
}

ed_status ro_reset(const Reorth* r, const LzScalars* S, const void* buf0, cudaStream_t s) {
  ED_TRY_CUDA(cudaMemsetAsync(r->F, 0, sizeof(RoFlags), s));
  ED_TRY_CUDA(cudaMemsetAsync(r->omega, 0, (size_t)3 * (r->slots + 2) * 8, s));
  // omega_{1,1} = 1 (array of step 1)
  const double one = 1.0;
  ED_TRY_CUDA(cudaMemcpyAsync(r->omega + (size_t)(1 % 3) * (r->slots + 2) + 1, &one, 8,
                              cudaMemcpyHostToDevice, s));
  return ro_store(r, S, 0, buf0, s);
}

ed_status ro_store(const Reorth* r, const LzScalars* S, int buf, const void* src, cudaStream_t s) {
  if (r->kind == 0)
    ro_store_t<float>(r, S, buf, src, s);
  else if (r->kind == 1)
    ro_store_t<double>(r, S, buf, src, s);
  else
    ro_store_t<long long>(r, S, buf, src, s);
  ED_TRY_CUDA(cudaGetLastError());
  return ED_OK;
}

template <typename T>
static void ro_passes_t(const Reorth* r, const LzScalars* S, void* Q, void* pb, int nb,
                        cudaStream_t s) {
  const size_t csm = (size_t)r->slots * 8;
  for (int pass = 0; pass < 2; ++pass) {
    ro_dots_kernel<T><<<r->G, kRoThreads, 0, s>>>(S, r->F, (const T*)Q, (const T*)r->V, r->n, r->part);
    ro_coef_kernel<<<r->slots, kRoThreads, 0, s>>>(S, r->F, r->kind, r->part, r->G, r->vscale, r->coef);
    ro_update_kernel<T><<<nb, kRoThreads, csm, s>>>(S, r->F, (T*)Q, (const T*)r->V, r->n, r->coef,
                                                    pass == 1, pb);
  }
}

ed_status ro_prepare(const Reorth* r) {
  const size_t csm = (size_t)r->slots * 8;
  if (csm > 48 * 1024) {
    if (r->kind == 0)
      ED_TRY_CUDA(allow_max_smem(ro_update_kernel<float>));
    else if (r->kind == 1)
      ED_TRY_CUDA(allow_max_smem(ro_update_kernel<double>));
    else
      ED_TRY_CUDA(allow_max_smem(ro_update_kernel<long long>));
  }
  return ED_OK;
}

// Between the update pass (q and its partial norms in pb, nb records) and the finish pass.
ed_status ro_apply(const Reorth* r, const LzScalars* S, void* Q, void* pb, int nb, cudaStream_t s) {
  if (r->mode == 3) return ED_OK;  // vectors are stored, never reorthogonalised
  ro_decide_kernel<<<1, kRoThreads, 0, s>>>(S, r->F, r->omega, r->mode, r->kind, pb, nb, r->slots,
                                            r->eps, r->psi);
  if (r->kind == 0)
    ro_passes_t<float>(r, S, Q, pb, nb, s);
  else if (r->kind == 1)
    ro_passes_t<double>(r, S, Q, pb, nb, s);
  else
    ro_passes_t<long long>(r, S, Q, pb, nb, s);
  ED_TRY_CUDA(cudaGetLastError());
  return ED_OK;
}

// psi[i] (rank order, FP64) = sum_{k < m} y[k + 1] s_k V_k[r ld + p] for the stored FP32
// vectors, with row r = i / cols, column c = i % cols at position p = colpos[c] (or c); the
// coefficients y_k s_k are rounded to FP32 and the sum is accumulated in FP32.
__global__ void __launch_bounds__(kRoThreads)
ro_ritz_f32_kernel(const double* __restrict__ y, int m, const float* __restrict__ V,
                   const double* __restrict__ vscale, int64_t n, int64_t dim, int64_t cols,
                   int64_t ld, const int32_t* __restrict__ colpos, double* __restrict__ psi) {
  extern __shared__ __align__(16) unsigned char ro_smem[];
  float* c = reinterpret_cast<float*>(ro_smem);
  for (int k = threadIdx.x; k < m; k += blockDim.x) c[k] = (float)(y[k + 1] * vscale[k]);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / cols, cc = i - r * cols;
    const int64_t e = r * ld + (colpos ? colpos[cc] : cc);
    float acc = 0.f;
    for (int k = 0; k < m; ++k) acc = fmaf(c[k], V[(int64_t)k * n + e], acc);
    psi[i] = (double)acc;
  }
}

ed_status ro_ritz_vector(const Reorth* r, const double* y, int m, int64_t dim, int64_t cols,
                         int64_t ld, const int32_t* colpos, double* psi, cudaStream_t s) {
  ED_CHECK_ARG(r->kind == 0, "internal: Ritz vectors are assembled from FP32 runs only");
  ED_CHECK_ARG(m >= 1 && m <= r->slots, "internal: Ritz vector of %d steps", m);
  int g = (int)((dim + kRoThreads - 1) / kRoThreads);
  const int cap = 4 * sm_count();
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  ro_ritz_f32_kernel<<<g, kRoThreads, (size_t)m * 4, s>>>(y, m, (const float*)r->V, r->vscale, r->n,
                                                           dim, cols, ld, colpos, psi);
  ED_TRY_CUDA(cudaGetLastError());
  return ED_OK;
}

ed_status ro_count(const Reorth* r, cudaStream_t s, int* count) {
  RoFlags f;
  ED_TRY_CUDA(cudaMemcpyAsync(&f, r->F, sizeof(f), cudaMemcpyDeviceToHost, s));
  ED_TRY_CUDA(cudaStreamSynchronize(s));
  *count = f.count;
  return ED_OK;
}

}  // namespace ed

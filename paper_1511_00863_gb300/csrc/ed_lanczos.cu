// Lanczos iteration (Sec. 2.2, Algorithm 1) on the device, the random start vector, and
// the lowest eigenvalue of the tridiagonal T by Sturm-sequence bisection in FP64.
//
// One step j is three launches on the run's stream:
//   1. fused H.v:  w = H f_j - b_j f_{j-1}, written over the f_{j-1} buffer, with per-CTA
//      partial sums of w . f_j  (ed_hv.cu, LzHvArgs);
//   2. update:     a_j = sum of the partials (every CTA sums them in the same order),
//      q = w - a_j f_j in place, per-CTA partial sums of q . q;
//   3. finish (one CTA): b_{j+1} = sqrt(sum), breakdown test, f_{j+1} = q / b_{j+1} kept
//      implicit as a buffer scale, E0(j) = lambda_min(T_j), convergence test.
// Each buffer holds an unnormalised vector B with f = scale * B, so no pass rescales it.
// Once the run stops (breakdown, convergence, max_steps) every later kernel returns at
// entry; ed_lanczos_solve replays a captured two-step CUDA graph and reads the status
// between batches of replays.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "ed_internal.cuh"
#include "ed_lanczos_dev.cuh"

namespace ed {


// ------------------------------------------------------------------ start vector
// SplitMix64 (Steele, Lea & Flood 2014): the (i+1)-th output of the generator seeded with
// `seed`; element i of the start vector is 2 * (top 53 bits * 2^-53) - 1.
__device__ __forceinline__ double start_element(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
}

// Partial sums of x_i^2 over the raw start vector.
__global__ void __launch_bounds__(kRedThreads)
start_norm_kernel(uint64_t seed, int64_t n, double* __restrict__ partial) {
  __shared__ double red[33];
  double v = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double e = start_element(seed, (uint64_t)i);
    v = fma(e, e, v);
  }
  v = block_sum(v, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

// Scalar i of the vector (row r = i / cols, column c = i % cols) goes to out[r ld + p] with
// p = cx colpos[c / cx] + c % cx (cx = 2 for the (re, im) scalars of a complex element) or
// p = c when colpos is NULL.
__device__ __forceinline__ int64_t col_of(const int32_t* colpos, int64_t c, int cx) {
  if (!colpos) return c;
  const int64_t e = c / cx;
  return cx * (int64_t)colpos[e] + (c - e * cx);
}

// out[row, col_of(c)] = raw_i / ||raw|| rounded to T.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
start_write_kernel(uint64_t seed, int64_t n, int64_t cols, int64_t ld, const int32_t* __restrict__ colpos,
                   int cx, const double* __restrict__ partial, int nparts, T* __restrict__ out) {
  __shared__ double red[33];
  const double inv = 1.0 / sqrt(block_sum_array(partial, nparts, red));
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / cols, c = i - r * cols;
    out[r * ld + col_of(colpos, c, cx)] = (T)(start_element(seed, (uint64_t)i) * inv);
  }
}

// Copy a dense caller vector into the padded layout and accumulate its squared norm.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
copy_in_kernel(const T* __restrict__ src, int64_t n, int64_t cols, int64_t ld,
               const int32_t* __restrict__ colpos, int cx, T* __restrict__ dst,
               double* __restrict__ partial) {
  __shared__ double red[33];
  DotAcc<T> acc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / cols, c = i - r * cols;
    const T v = src[i];
    dst[r * ld + col_of(colpos, c, cx)] = v;
    acc.add(v, v);
  }
  const double v = block_sum(acc.get(), red);
  if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

__global__ void init_scalars_kernel(LzScalars* S, const double* __restrict__ partial,
                                    int nparts, int use_partial) {
  __shared__ double red[33];
  double nrm2 = 1.0;
  if (use_partial) nrm2 = block_sum_array(partial, nparts, red);
  if (threadIdx.x == 0) S->scale[0] = 1.0 / sqrt(nrm2);
}

// ------------------------------------------------------------------ update
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
lz_update_kernel(LzScalars* S, int cur, const T* __restrict__ bcur, T* __restrict__ bprev,
                 int64_t n, const double* __restrict__ pa, int na, double* __restrict__ pb) {
  __shared__ double red[33];
  if (S->status != 0) return;
  const double a = block_sum_array(pa, na, red);
  const int j = S->j + 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) S->alpha[j] = a;
  const T coef = (T)(a * S->scale[cur]);
  DotAcc<T> acc;
  // n is a multiple of 32 (padded rows): 16-byte vectors of 16 / sizeof(T) elements
  constexpr int VE = 16 / sizeof(T);
  typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type Vec;
  const Vec* c4 = reinterpret_cast<const Vec*>(bcur);
  Vec* p4 = reinterpret_cast<Vec*>(bprev);
  const int64_t nv = n / VE;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv;
       i += (int64_t)gridDim.x * blockDim.x) {
    Vec w = p4[i];
    const Vec c = c4[i];
    T* wv = reinterpret_cast<T*>(&w);
    const T* cv = reinterpret_cast<const T*>(&c);
#pragma unroll
    for (int e = 0; e < VE; ++e) {
      const T q = wv[e] - coef * cv[e];
      wv[e] = q;
      acc.add(q, q);
    }
    p4[i] = w;
  }
  const double v = block_sum(acc.get(), red);
  if (threadIdx.x == 0) pb[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kRedThreads)
lz_finish_kernel(LzScalars* S, int cur, const double* __restrict__ pb, int nb) {
  __shared__ double red[33];
  __shared__ int stop_s;
  if (S->status != 0) return;
  const int j = S->j + 1;
  const double b2 = block_sum_array(pb, nb, red);
  if (threadIdx.x == 0) {
    const double beta = sqrt(b2);
    stop_s = finish_record_beta(S, j, beta);
    if (stop_s == 0) S->scale[1 - cur] = 1.0 / beta;
  }
  __syncthreads();
  finish_tail(S, j, stop_s);
}

__global__ void __launch_bounds__(kRedThreads)
lz_energy_kernel(const LzScalars* S, double* out) {
  const int j = S->j;
  if (j < 1) {
    if (threadIdx.x == 0) *out = NAN;
    return;
  }
  __shared__ double sturm_work[kSturmWork];
  const double E = sturm_lowest(S->alpha, S->beta, j, NAN, sturm_work);
  if (threadIdx.x == 0) *out = E;
}

// E0(i) = lambda_min(T_i) for i = 1 .. m - 1, block i - 1 for step i: the history of a run
// whose steps computed E0 only at the stop step (no convergence test). The steps' scalars are
// final, so the m - 1 bisections run side by side on as many SMs instead of one after each
// step on one SM (FP64 multisection: 4-9 rounds of ~9 us each on GB300).
__global__ void __launch_bounds__(kRedThreads)
lz_history_kernel(LzScalars* S, int m) {
  const int i = (int)blockIdx.x + 1;
  if (i >= m) return;
  __shared__ double sturm_work[kSturmWork];
  const double E = sturm_lowest(S->alpha, S->beta, i, NAN, sturm_work);
  if (threadIdx.x == 0) S->E0[i] = E;
}

// Eigenvector y of T_m for its lowest eigenvalue lam (tridiag_ritz_vector); one thread.
__global__ void lz_ritz_kernel(const LzScalars* S, int m, double lam, double* y, double* work) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  tridiag_ritz_vector(S->alpha, S->beta, m, lam, y, work);
}

static int red_grid(int64_t n) {
  const int64_t want = (n + kRedThreads - 1) / kRedThreads;
  const int64_t cap = (int64_t)sm_count() * 4;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace ed

using namespace ed;

struct ed_lanczos {
  const ed_basis* basis = nullptr;
  ed_opts opts{};
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t ld = 0;      // padded row stride (elements)
  int64_t n = 0;       // dim_up * ld
  size_t esize = 8;
  void* B[2] = {nullptr, nullptr};
  int cur = 0;         // buffer holding f_j
  LzScalars* S = nullptr;
  double* pa = nullptr;  // partials of the H.v pass
  double* pb = nullptr;  // partials of the update pass
  double* tmp = nullptr;
  int64_t npa = 0, npb = 0;
  int hv_grid = 0;
  bool stopped = false;
  double graph_t = 0.0, graph_U = 0.0;  // parameters the captured graph was made with
  bool fx = false;     // ED_F64: int64 fixed-point buffers (ed_fixed.cu)
  FxRun fxr{};
  Hv2Plan* plan = nullptr;  // fused H.v on the padded layout (ed_hv2.cu), if it fits
  Reorth* ro = nullptr;     // stored Lanczos vectors when opts.reorth != 0 (ed_reorth.cu)
  cudaGraphExec_t graph = nullptr;
};

static ed_status lz_launch_step(ed_lanczos* st, const ed_params* p, cudaStream_t s,
                                cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr) {
  const ed_basis* b = st->basis;
  const int c = st->cur;
  if (st->fx) {
    long long* const B[2] = {(long long*)st->B[0], (long long*)st->B[1]};
    ed_status r = fx_step(b, st->fxr, p->t, p->U, B, c, st->ld, st->S, (long long*)st->pa,
                          (long long*)st->pb, s, ev0, ev1, st->plan, st->ro);
    if (r == ED_OK) st->cur = 1 - c;
    return r;
  }
  LzHvArgs lz{st->S, c, st->pa};
  int grid = 0;
  ed_status r;
  if (ev0) ED_TRY_CUDA(cudaEventRecord(ev0, s));
  const ed_dtype dt = st->opts.dtype;
  if (st->plan) {
    grid = hv2_grid(st->plan);
    r = hv2_launch(st->plan, b, p->t, p->U, st->B[c], st->B[1 - c], st->S, c, st->pa, s);
  } else if (dt == ED_C32) {
    r = launch_hvc<float>(b, p->t, p->U, st->B[c], st->B[1 - c], st->ld, s, &lz, &grid);
  } else if (dt == ED_C64) {
    r = launch_hvc<double>(b, p->t, p->U, st->B[c], st->B[1 - c], st->ld, s, &lz, &grid);
  } else if (dt == ED_F64_NATIVE)
    r = launch_hv<double>(b, p->t, p->U, (const double*)st->B[c], (double*)st->B[1 - c], st->ld,
                          s, &lz, &grid);
  else
    r = launch_hv<float>(b, p->t, p->U, (const float*)st->B[c], (float*)st->B[1 - c], st->ld,
                         s, &lz, &grid);
  if (r != ED_OK) return r;
  if (ev1) ED_TRY_CUDA(cudaEventRecord(ev1, s));
  // the update works on scalars: a complex vector is 2 n of them (a_j, b_j are real)
  const int64_t ns = is_complex(dt) ? 2 * st->n : st->n;
  const int ug = red_grid(ns);
  if (dt == ED_F64_NATIVE || dt == ED_C64)
    lz_update_kernel<double><<<ug, kRedThreads, 0, s>>>(
        st->S, c, (const double*)st->B[c], (double*)st->B[1 - c], ns, st->pa, grid, st->pb);
  else
    lz_update_kernel<float><<<ug, kRedThreads, 0, s>>>(
        st->S, c, (const float*)st->B[c], (float*)st->B[1 - c], ns, st->pa, grid, st->pb);
  ED_TRY_CUDA(cudaGetLastError());
  if (st->ro && (r = ro_apply(st->ro, st->S, st->B[1 - c], st->pb, ug, s)) != ED_OK) return r;
  lz_finish_kernel<<<1, kRedThreads, 0, s>>>(st->S, c, st->pb, ug);
  ED_TRY_CUDA(cudaGetLastError());
  if (st->ro && (r = ro_store(st->ro, st->S, 1 - c, st->B[1 - c], s)) != ED_OK) return r;
  st->cur = 1 - c;
  return ED_OK;
}

// internal: also accept reorth = 3 (store the vectors without reorthogonalising; the FP32
// phase of ed_lanczos_solve_mixed)
static ed_status check_opts(const ed_opts* o, bool internal = false) {
  ED_CHECK_ARG(o != nullptr, "opts is NULL");
  ED_CHECK_ARG(o->max_steps >= 1 && o->max_steps <= ED_MAX_STEPS,
               "max_steps = %d outside [1, %d]", o->max_steps, ED_MAX_STEPS);
  ED_CHECK_ARG(o->dtype == ED_F64 || o->dtype == ED_F32 || o->dtype == ED_F64_NATIVE ||
                   is_complex(o->dtype),
               "unknown dtype %d", (int)o->dtype);
  ED_CHECK_ARG(o->reorth >= 0 && o->reorth <= (internal ? 3 : 2),
               "reorth = %d outside 0 (none), 1 (full), 2 (partial)", o->reorth);
  ED_CHECK_ARG(o->reorth == 0 || !is_complex(o->dtype),
               "reorthogonalisation is available for the real dtypes only");
  ED_CHECK_ARG(std::isfinite(o->tol), "tol is not finite");
  return ED_OK;
}

extern "C" ed_status ed_start_vector(int64_t dim, uint64_t seed, ed_dtype dtype, void* out,
                                     void* stream) {
  clear_error();
  ED_CHECK_ARG(dim >= 1, "ed_start_vector: dim < 1");
  ED_CHECK_ARG(out != nullptr && aligned16(out), "ed_start_vector: out NULL or not 16-byte aligned");
  ED_CHECK_ARG(dtype == ED_F64 || dtype == ED_F32 || dtype == ED_F64_NATIVE,
               "ed_start_vector: unknown dtype");
  cudaStream_t s = (cudaStream_t)stream;
  const int g = red_grid(dim);
  double* part = nullptr;
  ED_TRY_CUDA(cudaMallocAsync((void**)&part, g * sizeof(double), s));
  start_norm_kernel<<<g, kRedThreads, 0, s>>>(seed, dim, part);
  if (dtype != ED_F32)
    start_write_kernel<double><<<g, kRedThreads, 0, s>>>(seed, dim, dim, dim, nullptr, 1, part, g,
                                                         (double*)out);
  else
    start_write_kernel<float><<<g, kRedThreads, 0, s>>>(seed, dim, dim, dim, nullptr, 1, part, g,
                                                        (float*)out);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(part, s);
  if (e != cudaSuccess) {
    set_error("ed_start_vector: %s", cudaGetErrorString(e));
    return ED_ERR_CUDA;
  }
  return ED_OK;
}

// ------------------------------------------------------------------ no-allocation variant
// Scratch of ed_start_vector_noalloc: the per-CTA partial sums of the squared norm. One
// copy per device that loads the library, kept until the process exits; every call shares
// it, so calls that overlap on the GPU race. Each call writes all the slots it reads, so
// nothing needs clearing between calls.
constexpr int kNoAllocPartials = 4096;
static __device__ __align__(256) double g_start_partials[kNoAllocPartials];

// Device address of g_start_partials on the current device (in host code the symbol names
// a host-side stand-in, not device memory). Resolved once per device, with that device
// current, on the first call there.
static ed_status noalloc_scratch(double** out) {
  static std::mutex mu;
  static double* addr[64] = {nullptr};
  int dev = 0;
  ED_TRY_CUDA(cudaGetDevice(&dev));
  ED_CHECK_ARG(dev >= 0 && dev < 64, "ed_start_vector_noalloc: device ordinal %d not supported", dev);
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_start_partials);
    if (e != cudaSuccess || p == nullptr) {
      set_error("ed_start_vector_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return ED_ERR_CUDA;
    }
    addr[dev] = (double*)p;
  }
  *out = addr[dev];
  return ED_OK;
}

extern "C" ed_status ed_start_vector_noalloc(int64_t dim, uint64_t seed, ed_dtype dtype, void* out,
                                             void* stream) {
  clear_error();
  ED_CHECK_ARG(dim >= 1, "ed_start_vector_noalloc: dim < 1");
  ED_CHECK_ARG(out != nullptr && aligned16(out),
               "ed_start_vector_noalloc: out NULL or not 16-byte aligned");
  ED_CHECK_ARG(dtype == ED_F64 || dtype == ED_F32 || dtype == ED_F64_NATIVE,
               "ed_start_vector_noalloc: unknown dtype");
  const int g = red_grid(dim);
  ED_CHECK_ARG(g <= kNoAllocPartials,
               "ed_start_vector_noalloc: needs %d partial sums, the static scratch holds %d", g,
               kNoAllocPartials);
  double* part = nullptr;
  const ed_status r = noalloc_scratch(&part);
  if (r != ED_OK) return r;
  cudaStream_t s = (cudaStream_t)stream;
  start_norm_kernel<<<g, kRedThreads, 0, s>>>(seed, dim, part);
  if (dtype != ED_F32)
    start_write_kernel<double><<<g, kRedThreads, 0, s>>>(seed, dim, dim, dim, nullptr, 1, part, g,
                                                         (double*)out);
  else
    start_write_kernel<float><<<g, kRedThreads, 0, s>>>(seed, dim, dim, dim, nullptr, 1, part, g,
                                                        (float*)out);
  ED_TRY_CUDA(cudaGetLastError());
  return ED_OK;
}

extern "C" void ed_lanczos_destroy(ed_lanczos* st) {
  if (!st) return;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != st->device) cudaSetDevice(st->device);
  if (st->stream) cudaStreamSynchronize(st->stream);
  if (st->graph) cudaGraphExecDestroy(st->graph);
  if (st->plan) hv2_free(st->plan);
  if (st->ro) ro_free(st->ro);
  for (int i = 0; i < 2; ++i)
    if (st->B[i]) cudaFree(st->B[i]);
  if (st->S) cudaFree(st->S);
  if (st->pa) cudaFree(st->pa);
  if (st->pb) cudaFree(st->pb);
  if (st->tmp) cudaFree(st->tmp);
  if (prev != st->device) cudaSetDevice(prev);
  delete st;
}

// check_every: compute E0(j) in the finish kernel every this many steps; step_mode: the
// caller drives the loop, so only breakdown and max_steps stop the run (no tol test).
// Bases below this many states use the default fused H.v variant order: timing every
// variant would cost more than their solves.
constexpr int64_t kAutotuneMinDim = (int64_t)1 << 22;

static ed_status lz_alloc(const ed_basis* b, const ed_opts* o, cudaStream_t s, ed_lanczos** out) {
  *out = nullptr;
  ED_CHECK_ARG(b != nullptr, "basis is NULL");
  ed_status r = check_opts(o, true);
  if (r != ED_OK) return r;
  ED_CHECK_ARG(is_complex(o->dtype) || !b->has_tau(),
               "the lattice has complex amplitudes; use ED_C32 or ED_C64");
  ed_lanczos* st = new ed_lanczos();
  st->basis = b;
  st->opts = *o;
  cudaGetDevice(&st->device);
  st->stream = s;
  // bytes per element (a complex element is an (re, im) pair)
  st->esize = o->dtype == ED_F32 ? 4 : o->dtype == ED_C32 ? 8 : o->dtype == ED_C64 ? 16 : 8;
  st->fx = o->dtype == ED_F64;
  if (st->fx) st->fxr = fx_make(b);
  st->ld = (b->dn.dim + 31) / 32 * 32;
  bool split = false;  // the split-row kernel (its own row stride; no timing of variants)
  if (o->dtype == ED_F32 || o->dtype == ED_F64) {
    // rows longer than shared memory: the split-row fused H.v lays each row out as two
    // padded slices
    const int lds = hv2_split_ld(b, o->dtype == ED_F64 ? kHv2Fx : kHv2F32, o->schedule, s);
    if (lds > 0) {
      st->ld = lds;
      split = true;
    }
  }
  st->n = b->up.dim * st->ld;
  // partial sums: one double per CTA, or four int64 words per CTA on the fixed-point path
  st->npa = hv_max_grid(b) * (st->fx ? 4 : 1);
  st->npb = (int64_t)sm_count() * 4 * (st->fx ? 6 : 1);
  auto fail = [&](ed_status e) {
    ed_lanczos_destroy(st);
    return e;
  };
  for (int i = 0; i < 2; ++i) {
    if (cudaMalloc(&st->B[i], st->n * st->esize) != cudaSuccess) {
      set_error("Lanczos work vectors: out of device memory (%lld bytes each)",
                (long long)(st->n * st->esize));
      return fail(ED_ERR_OOM);
    }
  }
  if (o->reorth != 0) {
    const ed_status rr = ro_create(o->reorth, o->dtype, st->n, o->max_steps, b->dim, &st->ro);
    if (rr != ED_OK) return fail(rr);
  }
  if (cudaMalloc((void**)&st->S, sizeof(LzScalars)) != cudaSuccess ||
      cudaMalloc((void**)&st->pa, st->npa * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&st->pb, st->npb * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&st->tmp, 64) != cudaSuccess) {
    set_error("Lanczos scalars: out of device memory");
    return fail(ED_ERR_OOM);
  }
  if (o->dtype == ED_F32 || o->dtype == ED_F64 || o->dtype == ED_C32) {
    const int mode = st->fx ? kHv2Fx : o->dtype == ED_C32 ? kHv2C32 : kHv2F32;
    int sched = o->schedule;
    if (split) sched = st->fx ? 30 : 31;
    if (sched < 0) {
      // autotune once per basis and dtype: time every variant on this run's zeroed buffers
      int& tuned = b->tuned_kind[(int)o->dtype];
      if (tuned == 0 && b->dim < kAutotuneMinDim) tuned = -1;  // default variant order
      if (tuned == 0) {
        ED_TRY_CUDA(cudaMemsetAsync(st->S, 0, sizeof(LzScalars), s));
        for (int i = 0; i < 2; ++i) ED_TRY_CUDA(cudaMemsetAsync(st->B[i], 0, st->n * st->esize, s));
        int k = 0;
        ed_status tr = hv2_autotune(b, mode, (int)st->ld, st->B[0], st->B[1], st->S, st->pa, s, &k);
        if (tr != ED_OK) return fail(tr);
        tuned = k > 0 ? k : -1;
      }
      sched = tuned > 0 ? tuned : -1;
    }
    ed_status pr = hv2_build(b, mode, (int)st->ld, sched, s, &st->plan);
    if (pr != ED_OK) return fail(pr);
  }
  *out = st;
  return ED_OK;
}

// Start a run on an allocated state: zero both buffers (their pads must hold 0), load f_1
// (caller vector or seeded start vector) and the run's scalars. check_every: compute E0(j)
// every this many steps; step_mode: the caller drives the loop (no tol test).
static ed_status lz_reset(ed_lanczos* st, const ed_opts* o, const void* f1, int check_every,
                          bool step_mode) {
  const ed_basis* b = st->basis;
  cudaStream_t s = st->stream;
  ED_CHECK_ARG(f1 == nullptr || aligned16(f1), "f1 must be 16-byte aligned");
  st->opts = *o;
  st->stopped = false;
  for (int i = 0; i < 2; ++i) ED_TRY_CUDA(cudaMemsetAsync(st->B[i], 0, st->n * st->esize, s));
  LzScalars h;
  memset(&h, 0, sizeof(h));
  h.check_every = check_every < 1 ? 1 : check_every;
  h.max_steps = o->max_steps;
  h.tol = step_mode ? 0.0 : o->tol;
  h.scale[0] = 1.0;
  h.scale[1] = 0.0;
  for (int i = 0; i < ED_MAX_STEPS + 2; ++i) h.E0[i] = NAN;
  ED_TRY_CUDA(cudaMemcpyAsync(st->S, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  // a complex vector is seen as scalars: dim (re, im) pairs = 2 dim scalars, rows of 2 cols
  // scalars with stride 2 ld, so the real kernels below write the interleaved layout
  const int cx = is_complex(o->dtype) ? 2 : 1;
  const int64_t dim = cx * b->dim, cols = cx * b->dn.dim, lds = cx * st->ld;
  const bool dbl = o->dtype == ED_F64_NATIVE || o->dtype == ED_C64;
  const int g = red_grid(dim);
  ED_CHECK_ARG((int64_t)g <= st->npb, "internal: partial buffer too small");
  st->cur = 0;
  const int32_t* colpos = hv2_colpos(st->plan);  // NULL: rank order (general kernels)
  if (st->fx) {
    const ed_status r = f1 == nullptr
        ? fx_start(b, st->fxr, o->seed, (long long*)st->B[0], st->ld, colpos, st->S,
                   (long long*)st->pb, s)
        : fx_copy_in(b, st->fxr, (const double*)f1, (long long*)st->B[0], st->ld, colpos, st->S,
                     (long long*)st->pb, s);
    if (r != ED_OK || !st->ro) return r;
    return ro_reset(st->ro, st->S, st->B[0], s);
  }
  if (f1 == nullptr) {
    start_norm_kernel<<<g, kRedThreads, 0, s>>>(o->seed, dim, st->pb);
    if (dbl)
      start_write_kernel<double><<<g, kRedThreads, 0, s>>>(o->seed, dim, cols, lds, colpos, cx,
                                                           st->pb, g, (double*)st->B[0]);
    else
      start_write_kernel<float><<<g, kRedThreads, 0, s>>>(o->seed, dim, cols, lds, colpos, cx,
                                                          st->pb, g, (float*)st->B[0]);
    init_scalars_kernel<<<1, 32, 0, s>>>(st->S, st->pb, g, 0);
  } else {
    if (dbl)
      copy_in_kernel<double><<<g, kRedThreads, 0, s>>>((const double*)f1, dim, cols, lds,
                                                       colpos, cx, (double*)st->B[0], st->pb);
    else
      copy_in_kernel<float><<<g, kRedThreads, 0, s>>>((const float*)f1, dim, cols, lds,
                                                      colpos, cx, (float*)st->B[0], st->pb);
    init_scalars_kernel<<<1, kRedThreads, 0, s>>>(st->S, st->pb, g, 1);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("Lanczos init: %s", cudaGetErrorString(e));
    return ED_ERR_CUDA;
  }
  if (st->ro) return ro_reset(st->ro, st->S, st->B[0], s);
  return ED_OK;
}

static ed_status lz_init(const ed_basis* b, const ed_opts* o, const void* f1, cudaStream_t s,
                         int check_every, bool step_mode, ed_lanczos** out) {
  ed_lanczos* st = nullptr;
  ed_status r = lz_alloc(b, o, s, &st);
  if (r != ED_OK) return r;
  if ((r = lz_reset(st, o, f1, check_every, step_mode)) != ED_OK) {
    ed_lanczos_destroy(st);
    return r;
  }
  *out = st;
  return ED_OK;
}

extern "C" ed_status ed_lanczos_init(const ed_basis* b, const ed_opts* o, const void* f1,
                                     void* stream, ed_lanczos** out) {
  clear_error();
  ED_CHECK_ARG(out != nullptr, "ed_lanczos_init: out is NULL");
  *out = nullptr;
  {
    const ed_status rc = check_opts(o);
    if (rc != ED_OK) return rc;
  }
  ed_status r = lz_init(b, o, f1, (cudaStream_t)stream, ED_MAX_STEPS + 1, true, out);
  if (r == ED_OK)
    r = o->dtype == ED_F64 ? fx_prepare(b)
        : is_complex(o->dtype) ? hvc_prepare(b, o->dtype)
                               : hv_prepare(b, o->dtype);
  if (r != ED_OK && *out) {
    ed_lanczos_destroy(*out);
    *out = nullptr;
  }
  return r;
}

extern "C" ed_status ed_lanczos_step(ed_lanczos* st, const ed_params* p, double* alpha_j,
                                     double* beta_j1) {
  clear_error();
  ED_CHECK_ARG(st != nullptr && p != nullptr, "ed_lanczos_step: state or params is NULL");
  ED_CHECK_ARG(!st->stopped, "ed_lanczos_step: the run has stopped (breakdown or max_steps)");
  ed_status r = lz_launch_step(st, p, st->stream);
  if (r != ED_OK) return r;
  int hdr[2];
  ED_TRY_CUDA(cudaMemcpyAsync(hdr, st->S, 2 * sizeof(int), cudaMemcpyDeviceToHost, st->stream));
  ED_TRY_CUDA(cudaStreamSynchronize(st->stream));
  const int j = hdr[0], status = hdr[1];
  double ab[2] = {0, 0};
  ED_TRY_CUDA(cudaMemcpy(&ab[0], &st->S->alpha[j], sizeof(double), cudaMemcpyDeviceToHost));
  ED_TRY_CUDA(cudaMemcpy(&ab[1], &st->S->beta[j + 1], sizeof(double), cudaMemcpyDeviceToHost));
  if (alpha_j) *alpha_j = ab[0];
  if (beta_j1) *beta_j1 = ab[1];
  if (status != 0) st->stopped = true;
  return status == 1 ? ED_BREAKDOWN : ED_OK;
}

extern "C" ed_status ed_lanczos_run(ed_lanczos* st, const ed_params* p, int32_t nsteps,
                                    float* hv_ms) {
  clear_error();
  ED_CHECK_ARG(st != nullptr && p != nullptr, "ed_lanczos_run: state or params is NULL");
  ED_CHECK_ARG(nsteps >= 0 && nsteps <= ED_MAX_STEPS, "ed_lanczos_run: nsteps out of range");
  if (!hv_ms) {
    for (int i = 0; i < nsteps; ++i) {
      ed_status r = lz_launch_step(st, p, st->stream);
      if (r != ED_OK) return r;
    }
    return ED_OK;
  }
  std::vector<cudaEvent_t> ev(2 * (size_t)nsteps, nullptr);
  ed_status r = ED_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      set_error("ed_lanczos_run: event creation failed");
      r = ED_ERR_CUDA;
      break;
    }
  for (int i = 0; r == ED_OK && i < nsteps; ++i) r = lz_launch_step(st, p, st->stream, ev[2 * i], ev[2 * i + 1]);
  float total = 0.f;
  if (r == ED_OK && cudaStreamSynchronize(st->stream) != cudaSuccess) {
    set_error("ed_lanczos_run: %s", cudaGetErrorString(cudaGetLastError()));
    r = ED_ERR_CUDA;
  }
  for (int i = 0; r == ED_OK && i < nsteps; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) != cudaSuccess) {
      set_error("ed_lanczos_run: event timing failed");
      r = ED_ERR_CUDA;
    }
    total += ms;
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (r == ED_OK) *hv_ms = total;
  return r;
}

extern "C" ed_status ed_lanczos_buffers(const ed_lanczos* st, const void** f_next,
                                       const void** f_cur, double* scale_next,
                                       double* scale_cur, int64_t* ld, const int32_t** colpos) {
  clear_error();
  ED_CHECK_ARG(st != nullptr, "ed_lanczos_buffers: state is NULL");
  // after step j the buffer `cur` holds f_{j+1} (scale S->scale[cur]) and the other f_j
  double sc[2] = {0.0, 0.0};
  ED_TRY_CUDA(cudaMemcpyAsync(sc, st->S->scale, sizeof(sc), cudaMemcpyDeviceToHost, st->stream));
  ED_TRY_CUDA(cudaStreamSynchronize(st->stream));
  if (f_next) *f_next = st->B[st->cur];
  if (f_cur) *f_cur = st->B[1 - st->cur];
  if (scale_next) *scale_next = sc[st->cur];
  if (scale_cur) *scale_cur = sc[1 - st->cur];
  if (ld) *ld = st->ld;
  if (colpos) *colpos = hv2_colpos(st->plan);
  return ED_OK;
}

extern "C" ed_status ed_lanczos_schedule(const ed_lanczos* st, int32_t* schedule) {
  clear_error();
  ED_CHECK_ARG(st != nullptr && schedule != nullptr, "ed_lanczos_schedule: NULL argument");
  *schedule = st->plan ? hv2_kind(st->plan) : 0;
  return ED_OK;
}

extern "C" ed_status ed_lanczos_energy(ed_lanczos* st, double* E0, int32_t* steps) {
  clear_error();
  ED_CHECK_ARG(st != nullptr, "ed_lanczos_energy: state is NULL");
  lz_energy_kernel<<<1, kRedThreads, 0, st->stream>>>(st->S, st->tmp);
  ED_TRY_CUDA(cudaGetLastError());
  double e = 0;
  int j = 0;
  ED_TRY_CUDA(cudaMemcpyAsync(&e, st->tmp, sizeof(double), cudaMemcpyDeviceToHost, st->stream));
  ED_TRY_CUDA(cudaMemcpyAsync(&j, &st->S->j, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
  ED_TRY_CUDA(cudaStreamSynchronize(st->stream));
  if (E0) *E0 = e;
  if (steps) *steps = j;
  return ED_OK;
}

extern "C" ed_status ed_lanczos_ground_state(const ed_basis* b, const ed_params* p,
                                             const ed_opts* o, const void* f1, void* stream,
                                             double* psi, double* E0, int32_t* steps) {
  clear_error();
  ED_CHECK_ARG(b && p && o && psi && E0, "ed_lanczos_ground_state: NULL argument");
  ED_CHECK_ARG(o->dtype == ED_F64, "ed_lanczos_ground_state: dtype must be ED_F64");
  {
    const ed_status rc = check_opts(o);
    if (rc != ED_OK) return rc;
  }
  ED_CHECK_ARG(aligned16(psi), "ed_lanczos_ground_state: psi must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  ed_lanczos* st = nullptr;
  long long* P = nullptr;
  double* yd = nullptr;
  struct ReleaseOnReturn {  // frees the state and scratch on every return path
    ed_lanczos*& st;
    long long*& P;
    double*& yd;
    ~ReleaseOnReturn() {
      if (st) ed_lanczos_destroy(st);
      if (P) cudaFree(P);
      if (yd) cudaFree(yd);
    }
  } release{st, P, yd};
  // ---- pass 1: Algorithm 1 to convergence (stepwise, E0 every step)
  ed_status r = lz_init(b, o, f1, s, 1, false, &st);
  if (r != ED_OK) return r;
  if ((r = fx_prepare(b)) != ED_OK) return r;
  int hdr[2] = {0, 0};
  for (int done = 0; done < o->max_steps; done += 8) {
    for (int i = 0; i < 8; ++i)
      if ((r = lz_launch_step(st, p, s)) != ED_OK) return r;
    if (cudaMemcpyAsync(hdr, st->S, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("ed_lanczos_ground_state: %s", cudaGetErrorString(cudaGetLastError()));
      return ED_ERR_CUDA;
    }
    if (hdr[1] != 0) break;
  }
  const int m = hdr[0];
  const int status = hdr[1];
  double lam = 0.0;
  ED_TRY_CUDA(cudaMemcpy(&lam, &st->S->E0[m], sizeof(double), cudaMemcpyDeviceToHost));
  // ---- Ritz vector of T_m on the device
  if (cudaMalloc((void**)&yd, (size_t)(3 * (m + 2)) * sizeof(double)) != cudaSuccess)
    return ED_ERR_OOM;
  lz_ritz_kernel<<<1, 32, 0, s>>>(st->S, m, lam, yd, yd + (m + 2));
  ED_TRY_CUDA(cudaGetLastError());
  // ---- pass 2: the same steps again from the same start, accumulating y_j f_j
  ed_lanczos* st2 = nullptr;
  if ((r = lz_init(b, o, f1, s, ED_MAX_STEPS + 1, true, &st2)) != ED_OK) return r;
  ed_lanczos_destroy(st);
  st = st2;
  if (cudaMalloc((void**)&P, (size_t)b->dim * sizeof(long long)) != cudaSuccess)
    return ED_ERR_OOM;
  ED_TRY_CUDA(cudaMemsetAsync(P, 0, (size_t)b->dim * sizeof(long long), s));
  for (int j = 1; j <= m; ++j) {
    if ((r = fx_psi_accum(b, st->S, st->cur, yd, j, (const long long*)st->B[st->cur], st->ld,
                          hv2_colpos(st->plan), P, s)) != ED_OK)
      return r;
    if (j < m && (r = lz_launch_step(st, p, s)) != ED_OK) return r;
  }
  if ((r = fx_psi_finish(b, P, (long long*)st->pb, (double*)psi, s)) != ED_OK) return r;
  ED_TRY_CUDA(cudaStreamSynchronize(s));
  *E0 = lam;
  if (steps) *steps = m;
  if (status == 3 && o->tol > 0.0) {
    set_error("ed_lanczos_ground_state: not converged after %d steps", m);
    return ED_ERR_NOT_CONVERGED;
  }
  return ED_OK;
}

// ------------------------------------------------------------------ solve
// ed_lanczos_solve keeps, per basis, one allocated state per (dtype, schedule) and its
// instantiated two-step graph, so repeated solves skip allocation and capture; a solve that
// finds the cache busy (another thread) uses a private state instead.
struct SolveCache {
  std::mutex mu;
  cudaStream_t stream = nullptr;
  struct Entry {
    int dtype, schedule, reorth, slots;  // slots: stored vectors (reorth runs), else 0
    ed_lanczos* st;
  };
  std::vector<Entry> entries;
};
static std::mutex g_cache_mu;

namespace ed {
void lz_cache_free(const ed_basis* b) {
  SolveCache* C = (SolveCache*)b->solve_cache;
  if (!C) return;
  for (auto& e : C->entries) ed_lanczos_destroy(e.st);
  if (C->stream) cudaStreamDestroy(C->stream);
  delete C;
  b->solve_cache = nullptr;
}
}  // namespace ed

static ed_status solve_on(ed_lanczos* st, const ed_basis* b, const ed_params* p, const ed_opts* o,
                          const void* f1, double* E0, int32_t* steps, double* alpha, double* beta,
                          double* E0_hist) {
  cudaStream_t s = st->stream;
  // E0(j) every step when the convergence test needs it, else at the stop step (a history
  // is then computed after the run, all steps at once)
  const int check = o->tol > 0.0 ? 1 : ED_MAX_STEPS + 1;
  ed_status r = lz_reset(st, o, f1, check, false);
  if (r != ED_OK) return r;
  if ((r = (o->dtype == ED_F64 ? fx_prepare(b)
            : is_complex(o->dtype) ? hvc_prepare(b, o->dtype)
                                   : hv_prepare(b, o->dtype))) != ED_OK)
    return r;
  if (!st->graph || st->graph_t != p->t || st->graph_U != p->U) {
    if (st->graph) cudaGraphExecDestroy(st->graph);
    st->graph = nullptr;
    // capture two steps (the buffer roles alternate) and replay
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      set_error("ed_lanczos_solve: stream capture failed");
      return ED_ERR_CUDA;
    }
    const ed_status r1 = lz_launch_step(st, p, s);
    const ed_status r2 = r1 == ED_OK ? lz_launch_step(st, p, s) : r1;
    cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (r2 != ED_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (r2 == ED_OK) set_error("ed_lanczos_solve: capture failed: %s", cudaGetErrorString(ce));
      return r2 != ED_OK ? r2 : ED_ERR_CUDA;
    }
    ce = cudaGraphInstantiate(&st->graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
      st->graph = nullptr;
      set_error("ed_lanczos_solve: graph instantiate failed: %s", cudaGetErrorString(ce));
      return ED_ERR_CUDA;
    }
    st->graph_t = p->t;
    st->graph_U = p->U;
  }
  int hdr[2] = {0, 0};
  int launched = 0;
  while (true) {
    const int remaining = o->max_steps - launched;
    int batch = (remaining + 1) / 2;
    if (batch > 8) batch = 8;
    if (batch < 1) batch = 1;
    for (int i = 0; i < batch; ++i) ED_TRY_CUDA(cudaGraphLaunch(st->graph, s));
    launched += 2 * batch;
    ED_TRY_CUDA(cudaMemcpyAsync(hdr, st->S, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    ED_TRY_CUDA(cudaStreamSynchronize(s));
    if (hdr[1] != 0 || launched >= o->max_steps) break;
  }
  const int j = hdr[0];
  if (E0_hist && check > 1 && j > 1) {
    lz_history_kernel<<<j - 1, kRedThreads, 0, s>>>(st->S, j);
    ED_TRY_CUDA(cudaGetLastError());
  }
  std::vector<double> hv(3 * (size_t)(j + 2));
  double* h_alpha = hv.data();
  double* h_beta = h_alpha + (j + 2);
  double* h_E = h_beta + (j + 2);
  ED_TRY_CUDA(cudaMemcpyAsync(h_alpha, st->S->alpha, (j + 2) * 8, cudaMemcpyDeviceToHost, s));
  ED_TRY_CUDA(cudaMemcpyAsync(h_beta, st->S->beta, (j + 2) * 8, cudaMemcpyDeviceToHost, s));
  ED_TRY_CUDA(cudaMemcpyAsync(h_E, st->S->E0, (j + 2) * 8, cudaMemcpyDeviceToHost, s));
  ED_TRY_CUDA(cudaStreamSynchronize(s));
  *E0 = j >= 1 ? h_E[j] : NAN;
  if (steps) *steps = j;
  for (int i = 1; i <= j; ++i) {
    if (alpha) alpha[i - 1] = h_alpha[i];
    if (beta) beta[i - 1] = h_beta[i + 1];
    if (E0_hist) E0_hist[i - 1] = h_E[i];
  }
  const int status = hdr[1];
  if (status == 1) return ED_BREAKDOWN;
  if (status == 3 && o->tol > 0.0) {
    set_error("ed_lanczos_solve: not converged after %d steps", j);
    return ED_ERR_NOT_CONVERGED;
  }
  return ED_OK;
}

// Run fn(st) on the basis's cached state for opts o (allocated on first use), or on a
// private state when another thread holds the cache; the work is ordered after the work
// already queued on the caller's stream.
template <typename Fn>
static ed_status with_state(const ed_basis* b, const ed_opts* o, cudaStream_t user, Fn fn) {
  SolveCache* C = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (!b->solve_cache) {
      SolveCache* nc = new SolveCache();
      if (cudaStreamCreateWithFlags(&nc->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete nc;
        set_error("ed_lanczos_solve: stream creation failed");
        return ED_ERR_CUDA;
      }
      b->solve_cache = nc;
    }
    C = (SolveCache*)b->solve_cache;
  }
  std::unique_lock<std::mutex> lk(C->mu, std::try_to_lock);
  const bool cached = lk.owns_lock();
  cudaStream_t s = C->stream;
  if (!cached) ED_TRY_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t ev = nullptr;
  ED_TRY_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaEventRecord(ev, user);
  cudaStreamWaitEvent(s, ev, 0);
  cudaEventDestroy(ev);
  ed_lanczos* st = nullptr;
  ed_status r;
  if (cached) {
    const int slots = o->reorth ? o->max_steps : 0;
    for (auto& e : C->entries)
      if (e.dtype == (int)o->dtype && e.schedule == o->schedule && e.reorth == o->reorth &&
          e.slots >= slots)
        st = e.st;
    if (!st) {
      if ((r = lz_alloc(b, o, s, &st)) != ED_OK) return r;
      C->entries.push_back({(int)o->dtype, o->schedule, o->reorth, slots, st});
    }
    return fn(st);
  }
  if ((r = lz_alloc(b, o, s, &st)) != ED_OK) {
    cudaStreamDestroy(s);
    return r;
  }
  r = fn(st);
  ed_lanczos_destroy(st);
  cudaStreamDestroy(s);
  return r;
}

extern "C" ed_status ed_lanczos_solve(const ed_basis* b, const ed_params* p, const ed_opts* o,
                                      const void* f1, void* stream, double* E0, int32_t* steps,
                                      double* alpha, double* beta, double* E0_hist) {
  clear_error();
  ED_CHECK_ARG(b != nullptr && p != nullptr, "ed_lanczos_solve: basis or params is NULL");
  ED_CHECK_ARG(E0 != nullptr, "ed_lanczos_solve: E0 is NULL");
  ed_status r = check_opts(o);
  if (r != ED_OK) return r;
  return with_state(b, o, (cudaStream_t)stream, [&](ed_lanczos* st) {
    return solve_on(st, b, p, o, f1, E0, steps, alpha, beta, E0_hist);
  });
}

extern "C" ed_status ed_lanczos_solve_mixed(const ed_basis* b, const ed_params* p,
                                            const ed_opts* o, const void* f1,
                                            int32_t refine_steps, double refine_tol, void* stream,
                                            double* E0, int32_t* steps32, double* E0_fp32,
                                            int32_t* steps64, double* residual) {
  clear_error();
  ED_CHECK_ARG(b != nullptr && p != nullptr && o != nullptr && E0 != nullptr,
               "ed_lanczos_solve_mixed: NULL argument");
  ed_status r = check_opts(o);
  if (r != ED_OK) return r;
  ED_CHECK_ARG(o->dtype == ED_F32, "ed_lanczos_solve_mixed: opts->dtype must be ED_F32");
  ED_CHECK_ARG(o->reorth == 0, "ed_lanczos_solve_mixed: opts->reorth must be 0");
  ED_CHECK_ARG(refine_steps >= 1 && refine_steps <= ED_MAX_STEPS,
               "ed_lanczos_solve_mixed: refine_steps = %d outside [1, %d]", refine_steps,
               ED_MAX_STEPS);
  ED_CHECK_ARG(std::isfinite(refine_tol), "ed_lanczos_solve_mixed: refine_tol is not finite");
  ED_CHECK_ARG(!b->has_tau(), "ed_lanczos_solve_mixed: real lattices only");
  cudaStream_t user = (cudaStream_t)stream;
  // ---- FP32 phase: Algorithm 1 with the vectors kept, then the Ritz vector in rank order
  ed_opts o32 = *o;
  o32.reorth = 3;
  {
    // the FP32 phase keeps at most as many vectors as fit in half the free device memory
    // and in 96 GB; a shorter FP32 phase leaves more of the convergence to the refinement
    // steps
    size_t free_b = 0, total_b = 0;
    ED_TRY_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const double vbytes = (double)b->up.dim * (double)((b->dn.dim + 31) / 32 * 32) * 4.0;
    const double budget = std::min((double)free_b / 2.0, 96e9);
    const int cap = (int)std::min(budget / vbytes - 1.0, (double)ED_MAX_STEPS);
    ED_CHECK_ARG(cap >= 2, "ed_lanczos_solve_mixed: device memory for FP32 vectors too small");
    if (o32.max_steps > cap) o32.max_steps = cap;
    // beyond dim steps the FP32 recurrence only adds rounding noise
    if ((int64_t)o32.max_steps > b->dim) o32.max_steps = (int)std::max<int64_t>(b->dim, 1);
  }
  double* psi = nullptr;
  double* y = nullptr;
  int m = 0;
  double e32 = NAN;
  r = with_state(b, &o32, user, [&](ed_lanczos* st) -> ed_status {
    cudaStream_t s = st->stream;
    ed_status rr = solve_on(st, b, p, &o32, f1, &e32, &m, nullptr, nullptr, nullptr);
    if (rr < 0 && rr != ED_ERR_NOT_CONVERGED) return rr;
    if (m < 1) {
      set_error("ed_lanczos_solve_mixed: the FP32 phase took no step");
      return ED_ERR_ARG;
    }
    if (cudaMallocAsync((void**)&y, (size_t)3 * (m + 2) * sizeof(double), s) != cudaSuccess ||
        cudaMallocAsync((void**)&psi, (size_t)b->dim * sizeof(double), s) != cudaSuccess) {
      set_error("ed_lanczos_solve_mixed: out of device memory");
      return ED_ERR_OOM;
    }
    lz_ritz_kernel<<<1, 32, 0, s>>>(st->S, m, e32, y, y + (m + 2));
    ED_TRY_CUDA(cudaGetLastError());
    rr = ro_ritz_vector(st->ro, y, m, b->dim, b->dn.dim, st->ld, hv2_colpos(st->plan), psi, s);
    if (rr != ED_OK) return rr;
    ED_TRY_CUDA(cudaStreamSynchronize(s));
    return ED_OK;
  });
  auto release = [&](ed_status e) {
    if (y) cudaFreeAsync(y, user);
    if (psi) cudaFreeAsync(psi, user);
    return e;
  };
  if (r != ED_OK) return release(r);
  if (steps32) *steps32 = m;
  if (E0_fp32) *E0_fp32 = e32;
  // ---- FP64-accurate phase from psi: a_1 = psi.H psi (the Rayleigh quotient), b_2 = the
  // residual norm, E0 = lambda_min of the refined T
  ed_opts o64 = *o;
  o64.dtype = ED_F64;
  o64.max_steps = refine_steps;
  o64.tol = refine_tol;
  o64.schedule = -1;
  std::vector<double> a(refine_steps), bt(refine_steps);
  int32_t k = 0;
  r = with_state(b, &o64, user, [&](ed_lanczos* st) {
    return solve_on(st, b, p, &o64, psi, E0, &k, a.data(), bt.data(), nullptr);
  });
  if (r == ED_BREAKDOWN) r = ED_OK;
  if (steps64) *steps64 = k;
  if ((r == ED_OK || r == ED_ERR_NOT_CONVERGED) && residual) *residual = bt[0];
  return release(r);
}

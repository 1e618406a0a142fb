// Internal declarations shared by the libed translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>

#include "ed.h"
#include "ed_tables.h"  // hop-entry layout (kTargetMask, kSignBit)

namespace ed {

// Thread-local error message behind ed_last_error().
void set_error(const char* fmt, ...);
void clear_error();

#define ED_TRY_CUDA(call)                                                              \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      ::ed::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                      __LINE__);                                                       \
      return e_ == cudaErrorMemoryAllocation ? ED_ERR_OOM : ED_ERR_CUDA;               \
    }                                                                                  \
  } while (0)

#define ED_CHECK_ARG(cond, ...)      \
  do {                               \
    if (!(cond)) {                   \
      ::ed::set_error(__VA_ARGS__);  \
      return ED_ERR_ARG;             \
    }                                \
  } while (0)

constexpr int kMaxSites = 32;
constexpr int kBinomStride = 33;          // C[n * 33 + k], n, k in [0, 32]

// Hop table of one species: entry k of state r at hop[k * dim + r].
struct SpeciesTables {
  int64_t dim = 0;
  int32_t maxhops = 0;
  uint32_t* bits = nullptr;  // [dim]
  int32_t* hop = nullptr;    // [maxhops * dim], unused slots = dim
  // Lattices with per-bond amplitudes only: amplitude index of each hop, 2 b + 1 when the
  // state's particle sits at site j of bond b = (i, j) and hops to i, 2 b when it sits at i
  // and hops to j; same layout as `hop`.
  int32_t* hopa = nullptr;
};

}  // namespace ed

struct ed_basis {
  int device = 0;
  int32_t n_sites = 0, n_up = 0, n_dn = 0;
  int64_t dim = 0;
  ed::SpeciesTables up, dn;
  uint32_t* binom = nullptr;  // device copy of C(n, k), n, k <= 32
  // Order in which H.v kernels visit the up rows (reverse Cuthill-McKee order of the
  // up-species hop graph), so that rows sharing up-neighbours are processed close in
  // time and the neighbours stay resident in L2. NULL = rank order.
  int32_t* up_order = nullptr;
  // Workspaces of ed_lanczos_solve kept between calls (ed_lanczos.cu); freed with the basis.
  mutable void* solve_cache = nullptr;
  // Fused H.v variant chosen by timing for this basis, per dtype (0 = not tuned yet).
  mutable int tuned_kind[5] = {0, 0, 0, 0, 0};
  // Host-built down tables of the fused H.v per (V, G) geometry (ed_hv2.cu); freed with the
  // basis.
  mutable void* hv2_tables = nullptr;
  // Host-built split-row down tables (ed_hv2.cu), for rows longer than shared memory.
  mutable void* hv2_split = nullptr;
  // True when the caller's down species has a single state (N_dn = 0 or N_dn = n_sites) and
  // the up species more: the kernels then see the occupied species as the row (`dn`)
  // species, so a state vector is one row of C(L, N_up) elements instead of C(L, N_up) rows
  // padded to 32. The global index rank_up * dim_dn + rank_dn is unchanged (one factor is
  // 1); `up`/`dn` below are the kernels' view, user_up()/user_dn() the caller's.
  bool swapped = false;
  // Per-bond relative amplitudes (device, n_bonds (re, im) pairs) when the lattice has them;
  // then only the complex dtypes apply.
  int32_t n_bonds = 0;
  double2* tau = nullptr;
  bool has_tau() const { return tau != nullptr; }
  const ed::SpeciesTables& user_up() const { return swapped ? dn : up; }
  const ed::SpeciesTables& user_dn() const { return swapped ? up : dn; }
};

namespace ed {

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Row-staged H.v kernels run one CTA per few up rows; with fewer rows than this the
// element-parallel global kernels are chosen instead (automatic selection only).
constexpr int64_t kMinRowsStaged = 64;

// Number of SMs of the current device (cached per device).
int sm_count();
// Largest dynamic shared memory a CTA may opt in to on the current device (cached).
int smem_optin_max();
// Allow `kernel` the device's whole opt-in dynamic shared memory. The attribute is global
// to the kernel, not to a launch: setting it to one basis's need would make the captured
// graphs of a basis that needs more fail, so it is only ever raised to the maximum.
template <typename K>
inline cudaError_t allow_max_smem(K kernel) {
  cudaFuncAttributes fa;
  const cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  // the opt-in limit covers the kernel's static shared memory too
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_optin_max() - (int)fa.sharedSizeBytes);
}

// Free the solve workspaces cached on a basis (called by ed_basis_destroy).
void lz_cache_free(const ed_basis* b);
// Free the fused H.v down tables cached on a basis (called by ed_basis_destroy).
void hv2_tables_free(const ed_basis* b);

// Device-resident scalars of one Lanczos run (Algorithm 1). Index j is 1-based as in the
// paper: alpha[j] = a_j, beta[j] = b_j (beta[1] = 0), E0[j] = lambda_min(T_j).
// Buffer i of the run holds an unnormalised vector B_i with f = scale[i] * B_i.
struct LzScalars {
  int j;            // steps completed
  int status;       // 0 running, 1 breakdown, 2 converged, 3 max_steps reached
  int check_every;  // compute E0(j) every this many steps (and at the stop step)
  int max_steps;
  double tol;
  double tscale;    // max over i <= j of |a_i| + b_i (breakdown scale)
  double last_E0;   // most recent computed E0 and its step
  int last_E0_step;
  int pad_;
  double scale[2];
  // FP64-accurate (fixed-point) runs: buffer i holds int64 X_i with f = scale[i] * X_i.
  long long fx_max[2];          // max |X_i| of each buffer
  long long fx_a, fx_b, fx_c;   // H.v epilogue W = round((a S + b n X + c P) 2^fx_k)
  int fx_k, fx_r;               // ... and W's scale s_w = scale[cur] * 2^fx_r
  double fx_sw;
  double alpha[ED_MAX_STEPS + 2];
  double beta[ED_MAX_STEPS + 2];
  double E0[ED_MAX_STEPS + 2];
};

// Extra arguments of the Lanczos-fused H.v pass:
//   w = scale[cur] * H B_cur - b_j * scale[prev] * B_prev   (written over B_prev)
//   partial[block] = sum over the block's elements of w * (scale[cur] * B_cur)
struct LzHvArgs {
  const LzScalars* S;
  int cur;
  double* partial;
};

// Launch the H.v kernels: y = H x on rows of stride ld (ld >= dim_dn). T = float or double.
// With lz != nullptr, y must hold B_prev on entry and receives w (see LzHvArgs).
template <typename T>
ed_status launch_hv(const ed_basis* b, double t, double U, const T* x, T* y, int64_t ld,
                    cudaStream_t s, const LzHvArgs* lz = nullptr, int* grid_out = nullptr);

// Set the kernel attributes launch_hv relies on (dynamic shared memory size); call before
// the first launch on a device and outside stream capture.
ed_status hv_prepare(const ed_basis* b, ed_dtype dtype);

// Complex H.v (ed_hvc.cu) for ED_C32 (T = float) / ED_C64 (T = double): x, y are arrays of
// (re, im) pairs with row stride ld pairs; with lz, fused with the Lanczos epilogue like
// launch_hv (partial sums of the real dot product of the interleaved vectors).
template <typename T>
ed_status launch_hvc(const ed_basis* b, double t, double U, const void* x, void* y, int64_t ld,
                     cudaStream_t s, const LzHvArgs* lz = nullptr, int* grid_out = nullptr);
ed_status hvc_prepare(const ed_basis* b, ed_dtype dtype);
inline bool is_complex(ed_dtype d) { return d == ED_C32 || d == ED_C64; }

struct Reorth;  // stored Lanczos vectors for reorthogonalisation (ed_reorth.cu)

// FP64-accurate Lanczos path (int64 fixed point, ed_fixed.cu).
struct FxRun {
  int vb;      // vector bound exponent: |X| <= 2^vb
  int hops;    // maxhops_up + maxhops_dn
  int nmax;    // max doubly occupied sites = min(n_up, n_dn)
};
FxRun fx_make(const ed_basis* b);
// Start vector of SplitMix64 `seed` (exact in fixed point) into X (layout rows x ld, down
// rank d at column colpos[d], or d if colpos is NULL), and the run's initial scalars
// (scale[0], fx_max[0]). part: >= 4 * 4 * sm_count longs.
ed_status fx_start(const ed_basis* b, const FxRun& fx, uint64_t seed, long long* X, int64_t ld,
                   const int32_t* colpos, LzScalars* S, long long* part, cudaStream_t s);
// Caller FP64 vector f1 (dense, rank order) converted to fixed point (exponent from max |f1|).
ed_status fx_copy_in(const ed_basis* b, const FxRun& fx, const double* f1, long long* X,
                     int64_t ld, const int32_t* colpos, LzScalars* S, long long* part,
                     cudaStream_t s);
// One step of Algorithm 1 on the fixed-point buffers (cur holds f_j, the other f_{j-1}).
ed_status fx_step(const ed_basis* b, const FxRun& fx, double t, double U, long long* const B[2],
                  int cur, int64_t ld, LzScalars* S, long long* pa, long long* pb,
                  cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, const struct Hv2Plan* plan,
                  const Reorth* ro = nullptr);
ed_status fx_prepare(const ed_basis* b);
// Ground-state vector (ed_lanczos_ground_state): P += round(y_j scale[cur] 2^60 X_cur),
// and the final normalised, sign-gauged FP64 vector. part: >= 6 * 4 * sm_count longs.
ed_status fx_psi_accum(const ed_basis* b, const LzScalars* S, int cur, const double* y, int j,
                       const long long* X, int64_t ld, const int32_t* colpos, long long* P,
                       cudaStream_t s);
ed_status fx_psi_finish(const ed_basis* b, const long long* P, long long* part, double* out,
                        cudaStream_t s);

// Reorthogonalisation of the Lanczos residual (ed_reorth.cu; ed_opts.reorth 1 = full,
// 2 = partial): the run keeps every Lanczos vector on the device.
ed_status ro_create(int mode, ed_dtype dtype, int64_t n, int max_steps, int64_t dim, Reorth** out);
void ro_free(Reorth* r);
ed_status ro_prepare(const Reorth* r);
// Start of a run: clear the estimates, store f_1 (buffer 0).
ed_status ro_reset(const Reorth* r, const LzScalars* S, const void* buf0, cudaStream_t s);
// After the finish pass: store f_{j+1} (buffer buf, scale S->scale[buf]) in slot S->j.
ed_status ro_store(const Reorth* r, const LzScalars* S, int buf, const void* src, cudaStream_t s);
// Between the update pass (residual Q, its partial norm records pb[nb]) and the finish pass.
ed_status ro_apply(const Reorth* r, const LzScalars* S, void* Q, void* pb, int nb, cudaStream_t s);
// Number of steps reorthogonalised so far in the current run (synchronises s).
ed_status ro_count(const Reorth* r, cudaStream_t s, int* count);
// Ritz vector psi = sum_{k<m} y_{k+1} f_{k+1} of a run with stored FP32 vectors, written as
// a dense FP64 vector in rank order (y: device, 1-based; colpos: column of each down rank).
ed_status ro_ritz_vector(const Reorth* r, const double* y, int m, int64_t dim, int64_t cols,
                         int64_t ld, const int32_t* colpos, double* psi, cudaStream_t s);

// Lanczos-fused H.v on the library's padded vectors (ed_hv2.cu). hv2_build leaves *out
// NULL when no variant fits in shared memory (the general kernels are used then).
struct Hv2Plan;
// schedule: -1 = default variant, else a variant id (see ed_hv2.cu) if it fits.
// mode: kHv2F32 (FP32 vectors), kHv2Fx (int64 fixed point), kHv2C32 (complex FP32).
enum { kHv2F32 = 0, kHv2Fx = 1, kHv2C32 = 2 };
ed_status hv2_build(const ed_basis* b, int mode, int ld, int schedule, cudaStream_t s,
                    Hv2Plan** out);
void hv2_free(Hv2Plan* p);
int hv2_grid(const Hv2Plan* p);
// Row stride the fused H.v needs for this basis and precision when its rows only fit in
// shared memory as two slices (the split-row kernel), else 0 (the stride is then dim_dn
// rounded up to 32). Builds and caches the split tables on the basis.
// schedule 30 (int64) / 31 (FP32) asks for the split-row kernel whether or not rows fit.
int hv2_split_ld(const ed_basis* b, int mode, int schedule, cudaStream_t s);
// Column of each down rank in the plan's row layout (device, dim_dn entries).
const int32_t* hv2_colpos(const Hv2Plan* p);
int hv2_kind(const Hv2Plan* p);
// Time every fused H.v variant that fits on x (f_j) and y (f_{j-1} / w) with scalars S
// (zeroed: a neutral step) and return the fastest variant id (0 if none fits).
ed_status hv2_autotune(const ed_basis* b, int mode, int ld, void* x, void* y,
                       const LzScalars* S, void* partial, cudaStream_t s, int* kind);
ed_status hv2_launch(const Hv2Plan* p, const ed_basis* b, double t, double U, const void* x,
                     void* y, const LzScalars* S, int cur, void* partial, cudaStream_t s);

// Upper bound on the number of CTAs of any H.v launch of a Lanczos step (launch_hv,
// launch_hvc, the fixed-point kernels, the fused plans): the size of the partial-sum buffer.
int64_t hv_max_grid(const ed_basis* b);

// ---------------------------------------------------------------- reductions
// Dot-product accumulator: FP64 for FP64 data; for FP32 data an exact product (FMA
// error term) fed into a compensated FP32 pair, converted to FP64 once per thread.
template <typename T> struct DotAcc;
template <> struct DotAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ double get() const { return v; }
};
template <> struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float s = hi + p;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += err + e;
  }
  __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};

// Deterministic block sum (fixed shuffle tree, then warp 0 over the warp sums); the
// result is valid in thread 0. `sm` holds >= 32 doubles. Ends with a __syncthreads.
__device__ __forceinline__ double block_sum(double v, double* sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sm[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? sm[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;
}

// Sum of n partials in a fixed order by one block (every thread gets the result).
__device__ __forceinline__ double block_sum_array(const double* p, int64_t n, double* sm) {
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v += p[i];
  v = block_sum(v, sm);
  if (threadIdx.x == 0) sm[32] = v;
  __syncthreads();
  v = sm[32];
  __syncthreads();
  return v;
}

}  // namespace ed

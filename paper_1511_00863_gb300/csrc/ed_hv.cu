// y = H x for the tight-binding / Hubbard Hamiltonian (Sec. 1 Eq. 1 + on-site U), split
// as H = H_up (x) I + I (x) H_dn + D (Sec. 2.1 Eq. 3; Sec. 4 Eqs. 5-6).
//
// Layout: x[u * ld + d], u = up rank (slow), d = down rank (fast), ld >= dim_dn.
// Row-staged kernel: a CTA owns R consecutive up rows u0..u0+R-1. It copies those R rows
// of x into shared memory, interleaved as xs[d * R + r] (one extra zero slot at d = dim_dn
// absorbs the padding entries of the hop table), so that
//   * the down part  y[u,d] += -t s x[u, tgt_dn(d,k)]   gathers from shared memory and each
//     hop-table entry, read once, serves all R rows;
//   * the up part    y[u,d] += -t s x[tgt_up(u,k), d]   reads whole neighbouring rows,
//     coalesced along d (consecutive threads own consecutive d);
//   * the diagonal   y[u,d] += U popc(up[u] & dn[d]) x[u,d]   uses the integer popcount.
#include "ed_internal.cuh"

namespace ed {

constexpr int kHvThreads = 256;

struct HvArgs {
  const uint32_t* __restrict__ up_bits;
  const uint32_t* __restrict__ dn_bits;
  const int32_t* __restrict__ hop_up;
  const int32_t* __restrict__ hop_dn;
  int64_t dim_up, dim_dn, ld;
  int maxhops_up, maxhops_dn;
  double t, U;
};

// acc += c_k v_k over a state's hops in table order (c_k = -t or +t by the fermion sign; the
// same sequence of multiply-adds as a one-at-a-time loop, so the same rounding), taking the
// table entries and gathered values of four hops before adding any: more loads in flight.
// tab[k * stride] is hop k's entry; a target >= n is padding, and the rest of the state's
// list is padding too.
template <typename T, typename Load>
__device__ __forceinline__ void hv_add_hops(T& acc, const int32_t* tab, int64_t stride, int mh, int64_t n,
                                            T tt, Load load) {
  int k = 0;
  for (; k + 4 <= mh; k += 4) {
    uint32_t e[4];
    T v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) e[q] = (uint32_t)tab[(int64_t)(k + q) * stride];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t tg = (int64_t)(e[q] & kTargetMask);
      v[q] = tg < n ? load(tg) : T(0);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if ((int64_t)(e[q] & kTargetMask) < n) acc += ((e[q] & kSignBit) ? tt : -tt) * v[q];
    if ((int64_t)(e[3] & kTargetMask) >= n) return;
  }
  for (; k < mh; ++k) {
    const uint32_t e = (uint32_t)tab[(int64_t)k * stride];
    const int64_t tg = (int64_t)(e & kTargetMask);
    if (tg >= n) return;
    acc += ((e & kSignBit) ? tt : -tt) * load(tg);
  }
}

template <typename T, int R, bool kLz>
__global__ void __launch_bounds__(kHvThreads)
hv_staged_kernel(HvArgs a, const T* __restrict__ x, T* __restrict__ y, LzHvArgs lz) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[33];
  T sc = T(1), bsp = T(0);
  if (kLz) {
    if (lz.S->status != 0) return;
    const int j = lz.S->j + 1;
    sc = (T)lz.S->scale[lz.cur];
    bsp = (T)(lz.S->beta[j] * lz.S->scale[1 - lz.cur]);
  }
  DotAcc<T> dot;
  const int dn = (int)a.dim_dn;
  T* xs = reinterpret_cast<T*>(smem);
  int32_t* ut = reinterpret_cast<int32_t*>(xs + (size_t)(dn + 1) * R);
  const int64_t u0 = (int64_t)blockIdx.x * R;
  const T tt = (T)a.t, UU = (T)a.U;

#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t u = u0 + r;
    const T* xr = x + u * a.ld;
    for (int d = threadIdx.x; d < dn; d += blockDim.x) xs[d * R + r] = (u < a.dim_up) ? xr[d] : T(0);
  }
  if (threadIdx.x < R) xs[(size_t)dn * R + threadIdx.x] = T(0);
  for (int i = threadIdx.x; i < R * a.maxhops_up; i += blockDim.x) {
    const int r = i / a.maxhops_up, k = i - r * a.maxhops_up;
    const int64_t u = u0 + r;
    ut[i] = (u < a.dim_up) ? a.hop_up[(int64_t)k * a.dim_up + u] : (int32_t)a.dim_up;
  }
  uint32_t ub[R];
#pragma unroll
  for (int r = 0; r < R; ++r) ub[r] = (u0 + r < a.dim_up) ? a.up_bits[u0 + r] : 0u;
  __syncthreads();

  for (int d = threadIdx.x; d < dn; d += blockDim.x) {
    const uint32_t db = a.dn_bits[d];
    T acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = UU * (T)__popc(ub[r] & db) * xs[d * R + r];
    for (int k = 0; k < a.maxhops_dn; ++k) {
      const uint32_t e = (uint32_t)a.hop_dn[(int64_t)k * dn + d];
      const int tg = (int)(e & kTargetMask);
      const T c = (e & kSignBit) ? tt : -tt;
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] += c * xs[tg * R + r];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t u = u0 + r;
      if (u < a.dim_up) {
        hv_add_hops(acc[r], ut + r * a.maxhops_up, 1, a.maxhops_up, a.dim_up, tt,
                    [&](int64_t tg) { return x[tg * a.ld + d]; });
        if (kLz) {
          const T f = sc * xs[d * R + r];
          const T w = sc * acc[r] - bsp * y[u * a.ld + d];
          y[u * a.ld + d] = w;
          dot.add(w, f);
        } else {
          y[u * a.ld + d] = acc[r];
        }
      }
    }
  }
  if (kLz) {
    const double v = block_sum(dot.get(), red);
    if (threadIdx.x == 0) lz.partial[blockIdx.x] = v;
  }
}

// Fallback when a row does not fit in shared memory: one thread per element, every gather
// from global memory.
template <typename T, bool kLz>
__global__ void __launch_bounds__(kHvThreads)
hv_global_kernel(HvArgs a, const T* __restrict__ x, T* __restrict__ y, LzHvArgs lz) {
  __shared__ double red[33];
  T sc = T(1), bsp = T(0);
  if (kLz) {
    if (lz.S->status != 0) return;
    const int j = lz.S->j + 1;
    sc = (T)lz.S->scale[lz.cur];
    bsp = (T)(lz.S->beta[j] * lz.S->scale[1 - lz.cur]);
  }
  DotAcc<T> dot;
  const T tt = (T)a.t, UU = (T)a.U;
  const int64_t total = a.dim_up * a.dim_dn;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = g / a.dim_dn, d = g - u * a.dim_dn;
    const T* xr = x + u * a.ld;
    T acc = UU * (T)__popc(a.up_bits[u] & a.dn_bits[d]) * xr[d];
    hv_add_hops(acc, a.hop_dn + d, a.dim_dn, a.maxhops_dn, a.dim_dn, tt, [&](int64_t tg) { return xr[tg]; });
    hv_add_hops(acc, a.hop_up + u, a.dim_up, a.maxhops_up, a.dim_up, tt,
                [&](int64_t tg) { return x[tg * a.ld + d]; });
    if (kLz) {
      const T f = sc * xr[d];
      const T w = sc * acc - bsp * y[u * a.ld + d];
      y[u * a.ld + d] = w;
      dot.add(w, f);
    } else {
      y[u * a.ld + d] = acc;
    }
  }
  if (kLz) {
    const double v = block_sum(dot.get(), red);
    if (threadIdx.x == 0) lz.partial[blockIdx.x] = v;
  }
}

static HvArgs make_args(const ed_basis* b, double t, double U, int64_t ld) {
  HvArgs a;
  a.up_bits = b->up.bits;
  a.dn_bits = b->dn.bits;
  a.hop_up = b->up.hop;
  a.hop_dn = b->dn.hop;
  a.dim_up = b->up.dim;
  a.dim_dn = b->dn.dim;
  a.ld = ld;
  a.maxhops_up = b->up.maxhops;
  a.maxhops_dn = b->dn.maxhops;
  a.t = t;
  a.U = U;
  return a;
}

static int max_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

template <typename T, int R>
static size_t staged_smem(const ed_basis* b) {
  return (size_t)(b->dn.dim + 1) * R * sizeof(T) + (size_t)R * b->up.maxhops * sizeof(int32_t);
}

template <typename T, int R, bool kLz>
static ed_status launch_staged(const HvArgs& a, const ed_basis* b, const T* x, T* y,
                               cudaStream_t s, const LzHvArgs& lz, int* grid_out) {
  const size_t sm = staged_smem<T, R>(b);
  const int64_t grid = (b->up.dim + R - 1) / R;
  hv_staged_kernel<T, R, kLz><<<(unsigned)grid, kHvThreads, sm, s>>>(a, x, y, lz);
  ED_TRY_CUDA(cudaGetLastError());
  if (grid_out) *grid_out = (int)grid;
  return ED_OK;
}

static int global_grid(const ed_basis* b) {
  const int64_t want = (b->dim + kHvThreads - 1) / kHvThreads;
  const int64_t cap = (int64_t)sm_count() * 8;
  return (int)(want < cap ? want : cap);
}

template <typename T, bool kLz>
static ed_status launch_any(const ed_basis* b, const HvArgs& a, const T* x, T* y,
                            cudaStream_t s, const LzHvArgs& lz, int* grid_out) {
  const size_t lim = (size_t)max_smem_optin();
  const bool rows = b->up.dim >= kMinRowsStaged;
  if (rows && staged_smem<T, 2>(b) <= lim) return launch_staged<T, 2, kLz>(a, b, x, y, s, lz, grid_out);
  if (rows && staged_smem<T, 1>(b) <= lim) return launch_staged<T, 1, kLz>(a, b, x, y, s, lz, grid_out);
  const int grid = global_grid(b);
  hv_global_kernel<T, kLz><<<grid, kHvThreads, 0, s>>>(a, x, y, lz);
  ED_TRY_CUDA(cudaGetLastError());
  if (grid_out) *grid_out = grid;
  return ED_OK;
}

template <typename T>
ed_status launch_hv(const ed_basis* b, double t, double U, const T* x, T* y, int64_t ld,
                    cudaStream_t s, const LzHvArgs* lz, int* grid_out) {
  const HvArgs a = make_args(b, t, U, ld);
  if (lz) return launch_any<T, true>(b, a, x, y, s, *lz, grid_out);
  return launch_any<T, false>(b, a, x, y, s, LzHvArgs{nullptr, 0, nullptr}, grid_out);
}

template <typename T, int R>
static ed_status set_smem_attr(const ed_basis* b) {
  const int sm = (int)staged_smem<T, R>(b);
  ED_TRY_CUDA(allow_max_smem(hv_staged_kernel<T, R, false>));
  ED_TRY_CUDA(allow_max_smem(hv_staged_kernel<T, R, true>));
  return ED_OK;
}

template <typename T>
static ed_status prepare_t(const ed_basis* b) {
  const size_t lim = (size_t)max_smem_optin();
  if (staged_smem<T, 2>(b) <= lim && b->up.dim >= 2) return set_smem_attr<T, 2>(b);
  if (staged_smem<T, 1>(b) <= lim) return set_smem_attr<T, 1>(b);
  return ED_OK;
}

ed_status hv_prepare(const ed_basis* b, ed_dtype dtype) {
  return dtype == ED_F32 ? prepare_t<float>(b) : prepare_t<double>(b);
}

int64_t hv_max_grid(const ed_basis* b) {
  // row-staged kernels (real, complex, fixed point, fused): at most one CTA per up row;
  // element-parallel kernels of every path: at most 8 CTAs per SM (the fixed-point general
  // kernel launches twice its reduction grid, <= 2 x 4 per SM)
  const int64_t staged = b->up.dim;
  const int64_t g = (int64_t)sm_count() * 8;
  return staged > g ? staged : g;
}

template ed_status launch_hv<float>(const ed_basis*, double, double, const float*, float*,
                                    int64_t, cudaStream_t, const LzHvArgs*, int*);
template ed_status launch_hv<double>(const ed_basis*, double, double, const double*, double*,
                                     int64_t, cudaStream_t, const LzHvArgs*, int*);

}  // namespace ed

using namespace ed;

extern "C" ed_status ed_hv(const ed_basis* b, const ed_params* p, ed_dtype dtype, const void* x,
                           void* y, void* stream) {
  clear_error();
  ED_CHECK_ARG(b != nullptr && p != nullptr, "ed_hv: basis or params is NULL");
  ED_CHECK_ARG(x != nullptr && y != nullptr, "ed_hv: x or y is NULL");
  ED_CHECK_ARG(dtype == ED_F64 || dtype == ED_F32 || dtype == ED_F64_NATIVE || is_complex(dtype),
               "ed_hv: unknown dtype %d", (int)dtype);
  ED_CHECK_ARG(is_complex(dtype) || !b->has_tau(),
               "ed_hv: the lattice has complex amplitudes; use ED_C32 or ED_C64");
  ED_CHECK_ARG(aligned16(x) && aligned16(y), "ed_hv: x and y must be 16-byte aligned");
  const size_t es = dtype == ED_F32 ? 4 : dtype == ED_C32 ? 8 : dtype == ED_C64 ? 16 : 8;
  const char* xb = (const char*)x;
  const char* yb = (const char*)y;
  ED_CHECK_ARG(xb + b->dim * es <= yb || yb + b->dim * es <= xb, "ed_hv: x and y overlap");
  cudaStream_t s = (cudaStream_t)stream;
  if (is_complex(dtype)) {
    const ed_status rc = hvc_prepare(b, dtype);
    if (rc != ED_OK) return rc;
    return dtype == ED_C32 ? launch_hvc<float>(b, p->t, p->U, x, y, b->dn.dim, s)
                           : launch_hvc<double>(b, p->t, p->U, x, y, b->dn.dim, s);
  }
  const ed_status r = hv_prepare(b, dtype == ED_F32 ? ED_F32 : ED_F64_NATIVE);
  if (r != ED_OK) return r;
  if (dtype != ED_F32)
    return launch_hv<double>(b, p->t, p->U, (const double*)x, (double*)y, b->dn.dim, s);
  return launch_hv<float>(b, p->t, p->U, (const float*)x, (float*)y, b->dn.dim, s);
}

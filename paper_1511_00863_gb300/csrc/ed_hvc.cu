// Complex H.v for the complex dtypes (ED_C32, ED_C64): lattices with a relative complex
// amplitude tau_b per bond (Sec. 2.1: the checkerboard lattice's complex hoppings), or
// amplitude 1 on every bond when the lattice has none.
//
//   (H z)[g] = U popc(up & dn) z[g] + sum over the hops out of state g: A_h z[target]
// The states that hop into g are those reached by one hop out of g, and H[g, target] is
// the amplitude of the reverse hop, target -> g: if g's particle sits at j of bond
// b = (i, j) (the outgoing hop moves it to i), the reverse hop moves it from i to j (the
// conjugate term c+_j c_i), A_h = -t sign_h conj(tau_b); if it sits at i, A_h = -t sign_h
// tau_b.
//
// Same split as the real kernels (Sec. 2.1 Eq. 3, Sec. 4 Eqs. 5-6): a CTA stages R up rows
// of z in shared memory (down hops gather there; their table entries serve all R rows), up
// hops read neighbour rows coalesced along d. Complex elements are (re, im) pairs; the
// amplitude table (2 n_bonds entries, -t already applied) sits in shared memory. Fused with
// the Lanczos epilogue (kLz): w = s_cur H B_cur - b_j s_prev B_prev over B_prev, and per-CTA
// partial sums of Re(w . conj f_j) (the real dot product of the interleaved vectors), so
// the real Lanczos driver runs unchanged on 2 dim scalars.
#include "ed_internal.cuh"

namespace ed {

template <typename T>
struct CVec;
template <>
struct CVec<float> {
  typedef float2 type;
};
template <>
struct CVec<double> {
  typedef double2 type;
};

constexpr int kHvcThreads = 256;
constexpr int kMaxAmpShared = 8192;  // amplitude entries kept in shared memory

struct HvcArgs {
  const uint32_t* __restrict__ up_bits;
  const uint32_t* __restrict__ dn_bits;
  const int32_t* __restrict__ hop_up;
  const int32_t* __restrict__ hop_dn;
  const int32_t* __restrict__ hopa_up;  // NULL: every amplitude is -t
  const int32_t* __restrict__ hopa_dn;
  const double2* __restrict__ tau;      // NULL: every amplitude is -t
  int64_t dim_up, dim_dn, ld;
  int maxhops_up, maxhops_dn, namp;
  double t, U;
};

// a += b x (complex)
template <typename V>
__device__ __forceinline__ void cmac(V& a, const V& b, const V& x) {
  a.x = fma(b.x, x.x, fma(-b.y, x.y, a.x));
  a.y = fma(b.x, x.y, fma(b.y, x.x, a.y));
}

// Gather amplitude for hop-amplitude number i (2 b + 1: the state's particle sits at j of
// bond b; 2 b: at i): -t conj(tau_b) or -t tau_b, see the header; -t without per-bond
// amplitudes.
template <typename V>
__device__ __forceinline__ V amp_entry(const HvcArgs& a, int i) {
  V v;
  if (a.tau) {
    const double2 tb = a.tau[i >> 1];
    v.x = -a.t * tb.x;
    v.y = (i & 1) ? a.t * tb.y : -a.t * tb.y;
  } else {
    v.x = -a.t;
    v.y = 0.0;
  }
  return v;
}

template <typename V>
__device__ __forceinline__ V signed_amp(V A, uint32_t e) {
  if (e & kSignBit) {
    A.x = -A.x;
    A.y = -A.y;
  }
  return A;
}

// acc += A_k v_k over a state's hops in table order (the same complex multiply-adds as a
// one-at-a-time loop), taking the table entries and gathered values of four hops before
// adding any: more loads in flight. entry(k) gives hop k's table entry, amp(k, e) its signed
// amplitude, load(target) the gathered value; a target >= n is padding, and the rest of the
// state's list is padding too.
template <typename V, typename Entry, typename Amp, typename Load>
__device__ __forceinline__ void hvc_add_hops(V& acc, int mh, int64_t n, Entry entry, Amp amp, Load load) {
  int k = 0;
  for (; k + 4 <= mh; k += 4) {
    uint32_t e[4];
    V v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) e[q] = entry(k + q);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t tg = (int64_t)(e[q] & kTargetMask);
      if (tg < n) {
        v[q] = load(tg);
      } else {
        v[q].x = 0;
        v[q].y = 0;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if ((int64_t)(e[q] & kTargetMask) < n) cmac(acc, amp(k + q, e[q]), v[q]);
    if ((int64_t)(e[3] & kTargetMask) >= n) return;
  }
  for (; k < mh; ++k) {
    const uint32_t e = entry(k);
    const int64_t tg = (int64_t)(e & kTargetMask);
    if (tg >= n) return;
    cmac(acc, amp(k, e), load(tg));
  }
}

template <typename T, int R, bool kLz>
__global__ void __launch_bounds__(kHvcThreads)
hvc_staged_kernel(HvcArgs a, const typename CVec<T>::type* __restrict__ x,
                  typename CVec<T>::type* __restrict__ y, LzHvArgs lz) {
  typedef typename CVec<T>::type V;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[33];
  T sc = T(1), bsp = T(0);
  if (kLz) {
    if (lz.S->status != 0) return;
    const int j = lz.S->j + 1;
    sc = (T)lz.S->scale[lz.cur];
    bsp = (T)(lz.S->beta[j] * lz.S->scale[1 - lz.cur]);
  }
  const int dn = (int)a.dim_dn;
  const int MH = a.maxhops_up > 0 ? a.maxhops_up : 1;
  V* xs = reinterpret_cast<V*>(smem);                 // [(dn + 1) * R], zero slot at dn
  V* amp = xs + (size_t)(dn + 1) * R;                  // [namp]
  int32_t* ut = reinterpret_cast<int32_t*>(amp + a.namp);  // [R * MH] up targets
  int32_t* ua = ut + R * MH;                                // [R * MH] up amplitude numbers
  const int64_t u0 = (int64_t)blockIdx.x * R;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t u = u0 + r;
    for (int d = threadIdx.x; d <= dn; d += blockDim.x) {
      V v;
      v.x = T(0);
      v.y = T(0);
      if (d < dn && u < a.dim_up) v = x[u * a.ld + d];
      xs[(size_t)d * R + r] = v;
    }
  }
  for (int i = threadIdx.x; i < a.namp; i += blockDim.x) amp[i] = amp_entry<V>(a, i);
  for (int i = threadIdx.x; i < R * a.maxhops_up; i += blockDim.x) {
    const int r = i / a.maxhops_up, k = i - r * a.maxhops_up;
    const int64_t u = u0 + r;
    const bool ok = u < a.dim_up;
    ut[r * MH + k] = ok ? a.hop_up[(int64_t)k * a.dim_up + u] : (int32_t)a.dim_up;
    ua[r * MH + k] = (ok && a.hopa_up) ? a.hopa_up[(int64_t)k * a.dim_up + u] : 0;
  }
  __syncthreads();
  uint32_t ub[R];
#pragma unroll
  for (int r = 0; r < R; ++r) ub[r] = (u0 + r < a.dim_up) ? a.up_bits[u0 + r] : 0u;
  const T UU = (T)a.U;
  DotAcc<T> dot;
  for (int d = threadIdx.x; d < dn; d += blockDim.x) {
    V acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r].x = acc[r].y = T(0);
    for (int k = 0; k < a.maxhops_dn; ++k) {
      const uint32_t e = (uint32_t)a.hop_dn[(int64_t)k * a.dim_dn + d];
      const uint32_t tg = e & kTargetMask;
      if (tg >= (uint32_t)dn) break;
      const V A = signed_amp(amp[a.hopa_dn ? a.hopa_dn[(int64_t)k * a.dim_dn + d] : 0], e);
#pragma unroll
      for (int r = 0; r < R; ++r) cmac(acc[r], A, xs[(size_t)tg * R + r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      hvc_add_hops(
          acc[r], a.maxhops_up, a.dim_up, [&](int k) { return (uint32_t)ut[r * MH + k]; },
          [&](int k, uint32_t e) { return signed_amp(amp[ua[r * MH + k]], e); },
          [&](int64_t tg) { return x[tg * a.ld + d]; });
    }
    const uint32_t db = a.dn_bits[d];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t u = u0 + r;
      if (u >= a.dim_up) continue;
      const V xc = xs[(size_t)d * R + r];
      const T nU = UU * (T)__popc(ub[r] & db);
      V h;
      h.x = fma(nU, xc.x, acc[r].x);
      h.y = fma(nU, xc.y, acc[r].y);
      V* yp = y + u * a.ld + d;
      if (kLz) {
        const V P = *yp;
        V w;
        w.x = fma(sc, h.x, -bsp * P.x);
        w.y = fma(sc, h.y, -bsp * P.y);
        *yp = w;
        dot.add(w.x, sc * xc.x);
        dot.add(w.y, sc * xc.y);
      } else {
        *yp = h;
      }
    }
  }
  if (kLz) {
    const double v = block_sum(dot.get(), red);
    if (threadIdx.x == 0) lz.partial[blockIdx.x] = v;
  }
}

// One thread per element, every gather from global memory (rows too long for shared
// memory, or too few rows for the staged kernel).
template <typename T, bool kLz>
__global__ void __launch_bounds__(kHvcThreads)
hvc_global_kernel(HvcArgs a, const typename CVec<T>::type* __restrict__ x,
                  typename CVec<T>::type* __restrict__ y, LzHvArgs lz) {
  typedef typename CVec<T>::type V;
  __shared__ double red[33];
  T sc = T(1), bsp = T(0);
  if (kLz) {
    if (lz.S->status != 0) return;
    const int j = lz.S->j + 1;
    sc = (T)lz.S->scale[lz.cur];
    bsp = (T)(lz.S->beta[j] * lz.S->scale[1 - lz.cur]);
  }
  const T UU = (T)a.U;
  DotAcc<T> dot;
  const int64_t total = a.dim_up * a.dim_dn;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = g / a.dim_dn, d = g - u * a.dim_dn;
    const V* xr = x + u * a.ld;
    const V xc = xr[d];
    V acc;
    const T nU = UU * (T)__popc(a.up_bits[u] & a.dn_bits[d]);
    acc.x = nU * xc.x;
    acc.y = nU * xc.y;
    hvc_add_hops(
        acc, a.maxhops_dn, a.dim_dn, [&](int k) { return (uint32_t)a.hop_dn[(int64_t)k * a.dim_dn + d]; },
        [&](int k, uint32_t e) {
          return signed_amp(amp_entry<V>(a, a.hopa_dn ? a.hopa_dn[(int64_t)k * a.dim_dn + d] : 0), e);
        },
        [&](int64_t tg) { return xr[tg]; });
    hvc_add_hops(
        acc, a.maxhops_up, a.dim_up, [&](int k) { return (uint32_t)a.hop_up[(int64_t)k * a.dim_up + u]; },
        [&](int k, uint32_t e) {
          return signed_amp(amp_entry<V>(a, a.hopa_up ? a.hopa_up[(int64_t)k * a.dim_up + u] : 0), e);
        },
        [&](int64_t tg) { return x[tg * a.ld + d]; });
    V* yp = y + u * a.ld + d;
    if (kLz) {
      const V P = *yp;
      V w;
      w.x = fma(sc, acc.x, -bsp * P.x);
      w.y = fma(sc, acc.y, -bsp * P.y);
      *yp = w;
      dot.add(w.x, sc * xc.x);
      dot.add(w.y, sc * xc.y);
    } else {
      *yp = acc;
    }
  }
  if (kLz) {
    const double v = block_sum(dot.get(), red);
    if (threadIdx.x == 0) lz.partial[blockIdx.x] = v;
  }
}

// ------------------------------------------------------------------ host side
static HvcArgs hvc_args(const ed_basis* b, double t, double U, int64_t ld) {
  HvcArgs a;
  a.up_bits = b->up.bits;
  a.dn_bits = b->dn.bits;
  a.hop_up = b->up.hop;
  a.hop_dn = b->dn.hop;
  a.hopa_up = b->up.hopa;
  a.hopa_dn = b->dn.hopa;
  a.tau = b->tau;
  a.dim_up = b->up.dim;
  a.dim_dn = b->dn.dim;
  a.ld = ld;
  a.maxhops_up = b->up.maxhops;
  a.maxhops_dn = b->dn.maxhops;
  a.namp = b->has_tau() ? 2 * b->n_bonds : 1;
  if (a.namp < 1) a.namp = 1;
  a.t = t;
  a.U = U;
  return a;
}

template <typename T, int R>
static size_t hvc_smem(const ed_basis* b) {
  const int MH = b->up.maxhops > 0 ? b->up.maxhops : 1;
  const int namp = b->has_tau() ? (2 * b->n_bonds > 0 ? 2 * b->n_bonds : 1) : 1;
  return ((size_t)(b->dn.dim + 1) * R + namp) * sizeof(typename CVec<T>::type) + (size_t)R * MH * 8;
}

static int hvc_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// Rows staged per CTA (2, 1) or 0 for the element-parallel kernel.
template <typename T>
static int hvc_rows(const ed_basis* b) {
  if (b->up.dim < kMinRowsStaged) return 0;
  if (b->has_tau() && 2 * b->n_bonds > kMaxAmpShared) return 0;
  const size_t lim = (size_t)hvc_smem_optin();
  if (hvc_smem<T, 2>(b) <= lim) return 2;
  if (hvc_smem<T, 1>(b) <= lim) return 1;
  return 0;
}

static int hvc_global_grid(const ed_basis* b) {
  const int64_t want = (b->dim + kHvcThreads - 1) / kHvcThreads;
  const int64_t cap = (int64_t)sm_count() * 8;
  return (int)(want < cap ? want : cap);
}

template <typename T>
static ed_status hvc_prepare_t(const ed_basis* b) {
  const int R = hvc_rows<T>(b);
  if (R == 2) {
    ED_TRY_CUDA(allow_max_smem(hvc_staged_kernel<T, 2, true>));
    ED_TRY_CUDA(allow_max_smem(hvc_staged_kernel<T, 2, false>));
  } else if (R == 1) {
    ED_TRY_CUDA(allow_max_smem(hvc_staged_kernel<T, 1, true>));
    ED_TRY_CUDA(allow_max_smem(hvc_staged_kernel<T, 1, false>));
  }
  return ED_OK;
}

ed_status hvc_prepare(const ed_basis* b, ed_dtype dtype) {
  return dtype == ED_C32 ? hvc_prepare_t<float>(b) : hvc_prepare_t<double>(b);
}

template <typename T>
ed_status launch_hvc(const ed_basis* b, double t, double U, const void* x, void* y, int64_t ld,
                     cudaStream_t s, const LzHvArgs* lz, int* grid_out) {
  typedef typename CVec<T>::type V;
  const HvcArgs a = hvc_args(b, t, U, ld);
  const LzHvArgs none{nullptr, 0, nullptr};
  const int R = hvc_rows<T>(b);
  int grid;
  if (R > 0) {
    grid = (int)((b->up.dim + R - 1) / R);
    const size_t sm = R == 2 ? hvc_smem<T, 2>(b) : hvc_smem<T, 1>(b);
    if (R == 2) {
      if (lz) hvc_staged_kernel<T, 2, true><<<grid, kHvcThreads, sm, s>>>(a, (const V*)x, (V*)y, *lz);
      else hvc_staged_kernel<T, 2, false><<<grid, kHvcThreads, sm, s>>>(a, (const V*)x, (V*)y, none);
    } else {
      if (lz) hvc_staged_kernel<T, 1, true><<<grid, kHvcThreads, sm, s>>>(a, (const V*)x, (V*)y, *lz);
      else hvc_staged_kernel<T, 1, false><<<grid, kHvcThreads, sm, s>>>(a, (const V*)x, (V*)y, none);
    }
  } else {
    grid = hvc_global_grid(b);
    if (lz) hvc_global_kernel<T, true><<<grid, kHvcThreads, 0, s>>>(a, (const V*)x, (V*)y, *lz);
    else hvc_global_kernel<T, false><<<grid, kHvcThreads, 0, s>>>(a, (const V*)x, (V*)y, none);
  }
  ED_TRY_CUDA(cudaGetLastError());
  if (grid_out) *grid_out = grid;
  return ED_OK;
}

template ed_status launch_hvc<float>(const ed_basis*, double, double, const void*, void*, int64_t,
                                     cudaStream_t, const LzHvArgs*, int*);
template ed_status launch_hvc<double>(const ed_basis*, double, double, const void*, void*, int64_t,
                                      cudaStream_t, const LzHvArgs*, int*);

}  // namespace ed

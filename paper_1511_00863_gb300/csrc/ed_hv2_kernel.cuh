#pragma once
// Lanczos-fused H.v for the library's own (padded) vectors: the step that dominates a
// Lanczos iteration (Sec. 4: the product on the first line of Algorithm 1's loop).
//
//   w = s_cur H B_cur - b_j s_prev B_prev, written over B_prev, plus per-CTA partial sums
//   of w . f_j; H = H_up (x) I + I (x) H_dn + U D  (Sec. 2.1 Eq. 3, Sec. 4 Eqs. 5-6).
//
// Layout: B[u * ld + p], ld = dim_dn rounded up to 32 (pads hold 0 and stay 0). The column
// p of a row is not the down rank d itself: the plan orders the down states by their number
// of hops (most first; then by the number of hops with sign +1, most first; then by rank),
// p = colpos[d], so that the 32 V states a warp handles have (nearly) equal hop counts and
// the down loops run to the warp's own counts instead of the largest ones in the basis. The order is internal: vectors enter and leave the library
// in rank order (colpos is applied by the start, copy-in and ground-state kernels).
// One CTA owns R consecutive up rows; each thread owns V consecutive columns per iteration.
//  * The R rows are staged once into shared memory, interleaved so that one vector load
//    (R elements: 8 bytes for 2 x FP32, 16 bytes for 2 x int64) serves every row at once.
//    Column p goes to slot (p & ~(G-1)) | lo[p], lo a permutation inside each aligned group
//    of G = 128 / (R sizeof(E)) columns (G slots span all 32 banks, so slot mod G is the
//    bank group); the staging and epilogue accesses of a warp stay conflict-free. Slots
//    ld .. ld + G - 1 hold zeros, one per bank group.
//  * Down part: a per-plan table gives, for hop k of column p, the slot of the target
//    (16 bits); padding points at a zero slot. Within a chunk of 32 V columns (one warp) the
//    hops with fermion sign +1 come first and those with -1 after, each group padded to the
//    chunk's largest count, so the sign costs nothing per element; the columns are ordered
//    by (hop count, positive-hop count) to keep that padding small. The host chooses lo and
//    the order of each column's hops within its sign group (and the zero slot of each
//    padding entry) so that the G lanes of one shared-memory phase hit distinct bank groups
//    in as many steps as it can. Consecutive threads read consecutive table entries.
//  * Up part: each row's hop list is sorted by sign into shared memory once per CTA; the
//    threads then stream the neighbour rows with V-wide coalesced loads (L2-resident reuse).
//  * Diagonal: U popc(up[u] & dn[d]) x on the integer pipe.
// FP32 accumulates in FP32 (dot products compensated, FP64 per CTA). The int64 variant is
// the FP64-accurate path of ed_fixed.cu: exact hop sums, W = round((a S + b n X + c P) 2^k).
#include <cstring>

#include "ed_fixed.cuh"
#include "ed_internal.cuh"

namespace ed {

template <typename E, int N>
struct alignas(sizeof(E) * N) Pack {
  E v[N];
};

// Streaming (evict-first) access for the f_{j-1} / w stream, so the rows of f_j that
// neighbouring up rows will gather stay resident in L2.
template <typename E, int N>
__device__ __forceinline__ Pack<E, N> ldcs_pack(const Pack<E, N>* p) {
  Pack<E, N> r;
  if constexpr (sizeof(Pack<E, N>) == 16) {
    const int4 v = __ldcs(reinterpret_cast<const int4*>(p));
    memcpy(&r, &v, 16);
  } else if constexpr (sizeof(Pack<E, N>) == 8) {
    const long long v = __ldcs(reinterpret_cast<const long long*>(p));
    memcpy(&r, &v, 8);
  } else {
    const int v = __ldcs(reinterpret_cast<const int*>(p));
    memcpy(&r, &v, 4);
  }
  return r;
}
template <typename E, int N>
__device__ __forceinline__ void stcs_pack(Pack<E, N>* p, const Pack<E, N>& r) {
  if constexpr (sizeof(Pack<E, N>) == 16) {
    int4 v;
    memcpy(&v, &r, 16);
    __stcs(reinterpret_cast<int4*>(p), v);
  } else if constexpr (sizeof(Pack<E, N>) == 8) {
    long long v;
    memcpy(&v, &r, 8);
    __stcs(reinterpret_cast<long long*>(p), v);
  } else {
    int v;
    memcpy(&v, &r, 4);
    __stcs(reinterpret_cast<int*>(p), v);
  }
}

// Columns per aligned slot group: G slots of R elements cover the 32 banks once.
template <typename E, int R>
__host__ __device__ constexpr int hv2_group() {
  return 128 / (int)(sizeof(E) * R) < 32 ? 128 / (int)(sizeof(E) * R) : 32;
}

struct Hv2Args {
  const uint32_t* __restrict__ up_bits;
  const uint32_t* __restrict__ dn_bits;  // by column, padded to ld (pads 0)
  const uint16_t* __restrict__ dtab;     // [rows][ld] slot of the hop target
  const uchar2* __restrict__ kpn;        // per chunk of 32 V columns: positive, negative rows
  const uint8_t* __restrict__ slot_lo;   // [ld] slot of column p within its group of G
  const int32_t* __restrict__ hop_up;    // basis table [maxhops_up][dim_up]
  const int32_t* __restrict__ order;     // up-row visit order (NULL = rank order)
  int64_t dim_up;
  int ld, maxhops_up;
  float t, U;  // FP32 variant
};

template <typename E, int R, int V, int T, int MB>
__global__ void __launch_bounds__(T, MB)
hv2_kernel(Hv2Args a, const E* __restrict__ x, E* __restrict__ y, const LzScalars* __restrict__ S,
           int cur, void* __restrict__ partial) {
  constexpr int G = hv2_group<E, R>();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int npos_s[R], nneg_s[R];
  __shared__ double red[33];
  if (S->status != 0) return;
  const int ld = a.ld;
  const int MH = a.maxhops_up > 0 ? a.maxhops_up : 1;
  Pack<E, R>* xs = reinterpret_cast<Pack<E, R>*>(smem);
  int64_t* upoff = reinterpret_cast<int64_t*>(
      smem + ((size_t)(ld + G) * sizeof(Pack<E, R>) + 15) / 16 * 16);
  uint32_t* upraw = reinterpret_cast<uint32_t*>(upoff + R * MH);
  const int64_t g0 = (int64_t)blockIdx.x * R;
  int64_t urow[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t g = g0 + r;
    urow[r] = g < a.dim_up ? (a.order ? (int64_t)a.order[g] : g) : a.dim_up;  // dim_up = none
  }

  // ---- stage the R rows (one d per thread: R coalesced loads, one vector store); slots
  // ld .. ld + G - 1 are zero, one in each bank group
  for (int d = threadIdx.x; d < ld + G; d += T) {
    Pack<E, R> p;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t u = urow[r];
      p.v[r] = (d < ld && u < a.dim_up) ? x[u * ld + d] : E(0);
    }
    xs[d < ld ? (d & ~(G - 1)) | a.slot_lo[d] : d] = p;
  }
  // ---- up-hop lists: raw entries, then per row positives first, negatives after
  for (int i = threadIdx.x; i < R * a.maxhops_up; i += T) {
    const int r = i / a.maxhops_up, k = i - r * a.maxhops_up;
    int64_t u = a.dim_up;
#pragma unroll
    for (int rr = 0; rr < R; ++rr)
      if (rr == r) u = urow[rr];
    upraw[i] = (u < a.dim_up) ? (uint32_t)a.hop_up[(int64_t)k * a.dim_up + u] : (uint32_t)a.dim_up;
  }
  __syncthreads();
  if (threadIdx.x < R) {
    const int r = threadIdx.x;
    int np = 0, nn = 0;
    for (int k = 0; k < a.maxhops_up; ++k) {
      const uint32_t e = upraw[r * a.maxhops_up + k];
      const int64_t tg = (int64_t)(e & kTargetMask);
      if (tg >= a.dim_up) break;
      if (!(e & kSignBit)) upoff[r * MH + np++] = tg * ld;
    }
    for (int k = 0; k < a.maxhops_up; ++k) {
      const uint32_t e = upraw[r * a.maxhops_up + k];
      const int64_t tg = (int64_t)(e & kTargetMask);
      if (tg >= a.dim_up) break;
      if (e & kSignBit) upoff[r * MH + np + nn++] = tg * ld;
    }
    npos_s[r] = np;
    nneg_s[r] = nn;
  }
  __syncthreads();

  uint32_t ub[R];
  int npos[R], nneg[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    ub[r] = (urow[r] < a.dim_up) ? a.up_bits[urow[r]] : 0u;
    npos[r] = npos_s[r];
    nneg[r] = nneg_s[r];
  }
  // per-run scalars
  float sc = 1.f, bsp = 0.f;
  long long ca = 0, cb = 0, cc = 0;
  int ck = 0;
  if constexpr (sizeof(E) == 4) {
    const int j = S->j + 1;
    sc = (float)S->scale[cur];
    bsp = (float)(S->beta[j] * S->scale[1 - cur]);
  } else {
    ca = S->fx_a;
    cb = S->fx_b;
    cc = S->fx_c;
    ck = S->fx_k;
  }
  DotAcc<float> dotf;
  A192 dota;

  for (int d0 = threadIdx.x * V; d0 < ld; d0 += T * V) {
    E acc[R][V];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[r][v] = E(0);
    // ---- down part: gathers inside the staged rows. The chunk's table rows hold its
    // positive hops first (kpn.x rows), then its negative ones (kpn.y rows); padding points
    // at a zero slot.
    const uchar2 kpn = a.kpn[d0 / (32 * V)];
    const uint16_t* tp = a.dtab + d0;
    const int kend = kpn.x + kpn.y;
    if constexpr (sizeof(E) == 4) {
      // FP32: one loop, the sign as a warp-uniform +-1 factor of the FMA
#pragma unroll 2
      for (int k = 0; k < kend; ++k) {
        const Pack<uint16_t, V> e = *reinterpret_cast<const Pack<uint16_t, V>*>(tp + (size_t)k * ld);
        const float c = k < kpn.x ? 1.f : -1.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const Pack<E, R> q = xs[e.v[v]];
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r][v] = fmaf(c, q.v[r], acc[r][v]);
        }
      }
    } else {
      // int64: plain adds, then plain subtractions
      int k = 0;
#pragma unroll 2
      for (; k < kpn.x; ++k) {
        const Pack<uint16_t, V> e = *reinterpret_cast<const Pack<uint16_t, V>*>(tp + (size_t)k * ld);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const Pack<E, R> q = xs[e.v[v]];
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r][v] += q.v[r];
        }
      }
#pragma unroll 2
      for (; k < kend; ++k) {
        const Pack<uint16_t, V> e = *reinterpret_cast<const Pack<uint16_t, V>*>(tp + (size_t)k * ld);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const Pack<E, R> q = xs[e.v[v]];
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r][v] -= q.v[r];
        }
      }
    }
    // ---- up part: neighbouring rows, V-wide coalesced loads
    const E* xb = x + d0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t* uo = upoff + r * MH;
#pragma unroll 8
      for (int k = 0; k < npos[r]; ++k) {
        const Pack<E, V> q = *reinterpret_cast<const Pack<E, V>*>(xb + uo[k]);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[r][v] += q.v[v];
      }
#pragma unroll 4
      for (int k = 0; k < nneg[r]; ++k) {
        const Pack<E, V> q = *reinterpret_cast<const Pack<E, V>*>(xb + uo[npos[r] + k]);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[r][v] -= q.v[v];
      }
    }
    // ---- diagonal and the Lanczos epilogue
    const Pack<uint32_t, V> db = *reinterpret_cast<const Pack<uint32_t, V>*>(a.dn_bits + d0);
    const Pack<uint8_t, V> lo = *reinterpret_cast<const Pack<uint8_t, V>*>(a.slot_lo + d0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t u = urow[r];
      if (u >= a.dim_up) continue;
      E* yp = y + u * ld + d0;
      const Pack<E, V> P = ldcs_pack(reinterpret_cast<const Pack<E, V>*>(yp));
      Pack<E, V> W;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const E xc = xs[((d0 + v) & ~(G - 1)) | lo.v[v]].v[r];
        const int n = __popc(ub[r] & db.v[v]);
        if constexpr (sizeof(E) == 4) {
          const float hx = fmaf(-a.t, (float)acc[r][v], a.U * (float)n * (float)xc);
          const float w = fmaf(sc, hx, -bsp * (float)P.v[v]);
          W.v[v] = (E)w;
          dotf.add(w, sc * (float)xc);
        } else {
          const long long xi = (long long)xc;
          const W128 p = add128(add128(smul128(ca, (long long)acc[r][v]), smul128(cb, xi * n)),
                                smul128(cc, (long long)P.v[v]));
          const long long w = round_shift128(p, ck);
          W.v[v] = (E)w;
          a192_add_prod(dota, w, xi);
        }
      }
      stcs_pack(reinterpret_cast<Pack<E, V>*>(yp), W);
    }
  }
  if constexpr (sizeof(E) == 4) {
    const double v = block_sum(dotf.get(), red);
    if (threadIdx.x == 0) reinterpret_cast<double*>(partial)[blockIdx.x] = v;
  } else {
    // same record layout as the fixed-point reductions: (lo, lo >> 64, hi, max)
    __shared__ unsigned long long sm[32][3];
    I192 doti = a192_get(dota);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const I192 w = i192_shfl_down(doti, o);
      i192_add(doti, w);
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
      sm[wid][0] = (unsigned long long)doti.lo;
      sm[wid][1] = (unsigned long long)(doti.lo >> 64);
      sm[wid][2] = (unsigned long long)doti.hi;
    }
    __syncthreads();
    if (wid == 0) {
      I192 s;
      i192_zero(s);
      if (lane < T / 32) {
        s.lo = ((u128)sm[lane][1] << 64) | (u128)sm[lane][0];
        s.hi = (long long)sm[lane][2];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const I192 w = i192_shfl_down(s, o);
        i192_add(s, w);
      }
      if (lane == 0) {
        long long* out = reinterpret_cast<long long*>(partial) + 4 * blockIdx.x;
        out[0] = (long long)(unsigned long long)s.lo;
        out[1] = (long long)(unsigned long long)(s.lo >> 64);
        out[2] = s.hi;
        out[3] = 0;
      }
    }
  }
}

}  // namespace ed

// Lanczos-fused complex H.v (ED_C32: complex FP32 vectors) on the library's padded layout,
// the complex counterpart of hv2_kernel (ed_hv2_kernel.cuh) for lattices with per-bond
// amplitudes (Sec. 2.1: the checkerboard lattice's complex hoppings).
//
//   w = s_cur H B_cur - b_j s_prev B_prev over B_prev, partial sums of Re(w . conj f_j)
//
// Same plan as the real kernel: columns ordered by down-hop count with a per-chunk loop
// length, R up rows staged in shared memory (slot map against bank conflicts), V columns
// per thread. A down-table entry is 32 bits: the slot of the target (bits 0..15) and the
// index of its amplitude (bits 16..31) in a table of signed amplitudes kept in shared
// memory: index 2 a + s, a the hop's amplitude number (2 b + 1 when the state's particle
// sits at j of bond b = (i, j), else 2 b; 0 without per-bond amplitudes), s its fermion
// sign bit; value (-1)^s times the gather amplitude -t conj(tau_b) or -t tau_b (see
// ed_hvc.cu). Up-hop lists (neighbour row offset, amplitude index) per row in shared memory.
#pragma once

#include "ed_hv2_kernel.cuh"

namespace ed {

struct Hv2cArgs {
  const uint32_t* __restrict__ up_bits;
  const uint32_t* __restrict__ dn_bits;  // by column, padded to ld (pads 0)
  const uint32_t* __restrict__ dtab;     // [rows][ld] slot | amplitude index << 16
  const uchar2* __restrict__ kpn;        // per chunk of 32 V columns: loop length in .x
  const uint8_t* __restrict__ slot_lo;   // [ld] slot of column p within its group of G
  const int32_t* __restrict__ hop_up;    // basis table [maxhops_up][dim_up]
  const int32_t* __restrict__ hopa_up;   // amplitude numbers of the up hops (NULL: 0)
  const int32_t* __restrict__ order;     // up-row visit order (NULL = rank order)
  const double2* __restrict__ tau;       // per-bond relative amplitudes (NULL: all 1)
  int64_t dim_up;
  int ld, maxhops_up, namp;  // namp = 4 n_bonds with tau, else 2
  float t, U;
};

// Signed gather amplitude number i of the table (see the header).
__device__ __forceinline__ float2 hv2c_amp(const Hv2cArgs& a, int i) {
  const int num = i >> 1;
  float2 v;
  if (a.tau) {
    const double2 tb = a.tau[num >> 1];
    v.x = (float)(-(double)a.t * tb.x);
    v.y = (float)((num & 1) ? (double)a.t * tb.y : -(double)a.t * tb.y);
  } else {
    v = make_float2(-a.t, 0.f);
  }
  if (i & 1) v = make_float2(-v.x, -v.y);
  return v;
}

__device__ __forceinline__ void cmacf(float2& a, const float2& b, const float2& x) {
  a.x = fmaf(b.x, x.x, fmaf(-b.y, x.y, a.x));
  a.y = fmaf(b.x, x.y, fmaf(b.y, x.x, a.y));
}

template <int R, int V, int T, int MB>
__global__ void __launch_bounds__(T, MB)
hv2c_kernel(Hv2cArgs a, const float2* __restrict__ x, float2* __restrict__ y,
            const LzScalars* __restrict__ S, int cur, double* __restrict__ partial) {
  constexpr int G = hv2_group<float2, R>();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[33];
  if (S->status != 0) return;
  const int ld = a.ld;
  const int MH = a.maxhops_up > 0 ? a.maxhops_up : 1;
  Pack<float2, R>* xs = reinterpret_cast<Pack<float2, R>*>(smem);
  float2* amp = reinterpret_cast<float2*>(xs + (ld + G));
  int64_t* upoff = reinterpret_cast<int64_t*>(amp + ((a.namp + 1) & ~1));
  int32_t* upamp = reinterpret_cast<int32_t*>(upoff + R * MH);
  __shared__ int nup_s[R];
  const int64_t g0 = (int64_t)blockIdx.x * R;
  int64_t urow[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t g = g0 + r;
    urow[r] = g < a.dim_up ? (a.order ? (int64_t)a.order[g] : g) : a.dim_up;
  }
  // ---- stage the R rows into their slots (zero slots ld .. ld + G - 1), the amplitude
  // table, the up-hop lists
  for (int d = threadIdx.x; d < ld + G; d += T) {
    Pack<float2, R> p;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t u = urow[r];
      p.v[r] = (d < ld && u < a.dim_up) ? x[u * ld + d] : make_float2(0.f, 0.f);
    }
    xs[d < ld ? (d & ~(G - 1)) | a.slot_lo[d] : d] = p;
  }
  for (int i = threadIdx.x; i < a.namp; i += T) amp[i] = hv2c_amp(a, i);
  for (int i = threadIdx.x; i < R * a.maxhops_up; i += T) {
    const int r = i / a.maxhops_up, k = i - r * a.maxhops_up;
    int64_t u = a.dim_up;
#pragma unroll
    for (int rr = 0; rr < R; ++rr)
      if (rr == r) u = urow[rr];
    int64_t off = -1;
    int32_t ai = 0;
    if (u < a.dim_up) {
      const uint32_t e = (uint32_t)a.hop_up[(int64_t)k * a.dim_up + u];
      const int64_t tg = (int64_t)(e & kTargetMask);
      if (tg < a.dim_up) {
        off = tg * ld;
        const int32_t num = a.hopa_up ? a.hopa_up[(int64_t)k * a.dim_up + u] : 0;
        ai = 2 * num + (int32_t)(e >> 31);
      }
    }
    upoff[r * MH + k] = off;
    upamp[r * MH + k] = ai;
  }
  __syncthreads();
  if (threadIdx.x < R) {  // hops of a state come first in its list: count them
    int n = 0;
    while (n < a.maxhops_up && upoff[threadIdx.x * MH + n] >= 0) ++n;
    nup_s[threadIdx.x] = n;
  }
  __syncthreads();
  uint32_t ub[R];
  int nup[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    ub[r] = (urow[r] < a.dim_up) ? a.up_bits[urow[r]] : 0u;
    nup[r] = nup_s[r];
  }
  const int j = S->j + 1;
  const float sc = (float)S->scale[cur];
  const float bsp = (float)(S->beta[j] * S->scale[1 - cur]);
  DotAcc<float> dot;

  for (int d0 = threadIdx.x * V; d0 < ld; d0 += T * V) {
    float2 acc[R][V];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[r][v] = make_float2(0.f, 0.f);
    // ---- down part: gathers inside the staged rows
    const int kc = a.kpn[d0 / (32 * V)].x;
    const uint32_t* tp = a.dtab + d0;
#pragma unroll 2
    for (int k = 0; k < kc; ++k) {
      const Pack<uint32_t, V> e = *reinterpret_cast<const Pack<uint32_t, V>*>(tp + (size_t)k * ld);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const Pack<float2, R> q = xs[e.v[v] & 0xFFFFu];
        const float2 A = amp[e.v[v] >> 16];
#pragma unroll
        for (int r = 0; r < R; ++r) cmacf(acc[r][v], A, q.v[r]);
      }
    }
    // ---- up part: neighbouring rows, V-wide coalesced loads
    const float2* xb = x + d0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t* uo = upoff + r * MH;
      const int32_t* ua = upamp + r * MH;
#pragma unroll 4
      for (int k = 0; k < nup[r]; ++k) {
        const Pack<float2, V> q = *reinterpret_cast<const Pack<float2, V>*>(xb + uo[k]);
        const float2 A = amp[ua[k]];
#pragma unroll
        for (int v = 0; v < V; ++v) cmacf(acc[r][v], A, q.v[v]);
      }
    }
    // ---- diagonal and the Lanczos epilogue
    const Pack<uint32_t, V> db = *reinterpret_cast<const Pack<uint32_t, V>*>(a.dn_bits + d0);
    const Pack<uint8_t, V> lo = *reinterpret_cast<const Pack<uint8_t, V>*>(a.slot_lo + d0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t u = urow[r];
      if (u >= a.dim_up) continue;
      float2* yp = y + u * ld + d0;
      const Pack<float2, V> P = *reinterpret_cast<const Pack<float2, V>*>(yp);
      Pack<float2, V> W;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const float2 xc = xs[((d0 + v) & ~(G - 1)) | lo.v[v]].v[r];
        const float nU = a.U * (float)__popc(ub[r] & db.v[v]);
        const float hx = fmaf(nU, xc.x, acc[r][v].x), hy = fmaf(nU, xc.y, acc[r][v].y);
        const float wx = fmaf(sc, hx, -bsp * P.v[v].x), wy = fmaf(sc, hy, -bsp * P.v[v].y);
        W.v[v] = make_float2(wx, wy);
        dot.add(wx, sc * xc.x);
        dot.add(wy, sc * xc.y);
      }
      *reinterpret_cast<Pack<float2, V>*>(yp) = W;
    }
  }
  const double v = block_sum(dot.get(), red);
  if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

}  // namespace ed

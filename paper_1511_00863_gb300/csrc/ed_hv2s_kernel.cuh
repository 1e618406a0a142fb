#pragma once
// Lanczos-fused H.v for rows longer than shared memory (split rows): the same product and
// epilogue as hv2_kernel (Sec. 4, Eqs. 5-6; w = s_cur H B_cur - b_j s_prev B_prev written
// over B_prev, per-CTA partial sums of w . f_j), for bases whose down row (dim_dn elements)
// does not fit in one CTA's shared memory, e.g. the FP64-accurate 18-site 9/9 basis (389 KB
// rows of int64).
//
// The down states are cut in two slices by the occupation of one site (SplitTables): a hop
// changes that occupation only when it moves a particle onto or off the site, so most down
// hops stay inside their slice. One CTA owns one up row and processes it slice by slice. A
// slice is laid out and staged exactly like a whole row of hv2_kernel (R = 1): column order
// by hop count, slot map (p & ~(G-1)) | lo[p] against bank conflicts, zero slots ld_s ..
// ld_s + G - 1, per-lane hop order chosen by the host. The in-slice down hops gather from
// shared memory; the few cross-slice ones have table rows of their own and read the row in
// global memory (it is L2-resident while the CTA works on it); the up part streams the
// neighbour rows' columns of the slice; the epilogue is hv2_kernel's.
#include "ed_hv2_kernel.cuh"

namespace ed {

struct Hv2sArgs {
  const uint32_t* __restrict__ up_bits;
  const uint32_t* __restrict__ dn_bits;  // by column, padded (pads 0)
  const uint16_t* __restrict__ dtab;     // [rows][ld]: slot of the target inside the slice
  const uint16_t* __restrict__ xtab;     // [xrows][ld]: target column inside the other slice
  const uchar4* __restrict__ kpn;        // per chunk of 32 V columns: in +, in -, cross +, cross -
  const uint8_t* __restrict__ slot_lo;   // [ld] slot of column p within its group of G
  const int32_t* __restrict__ hop_up;    // basis table [maxhops_up][dim_up]
  const int32_t* __restrict__ order;     // up-row visit order (NULL = rank order)
  int64_t dim_up;
  int ld, maxhops_up, nslots;            // nslots: longest slice + G
  int cstart0, cstart1, cstart2;         // slices [cstart0, cstart1), [cstart1, cstart2)
  float t, U;                            // FP32 variant
};

template <typename E, int V, int T, int MB>
__global__ void __launch_bounds__(T, MB)
hv2s_kernel(Hv2sArgs a, const E* __restrict__ x, E* __restrict__ y,
            const LzScalars* __restrict__ S, int cur, void* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int npos_s, nneg_s;
  __shared__ double red[33];
  if (S->status != 0) return;
  const int ld = a.ld;
  const int MH = a.maxhops_up > 0 ? a.maxhops_up : 1;
  constexpr int G = hv2_group<E, 1>();
  E* xs = reinterpret_cast<E*>(smem);
  int64_t* upoff = reinterpret_cast<int64_t*>(smem + ((size_t)a.nslots * sizeof(E) + 15) / 16 * 16);
  uint32_t* upraw = reinterpret_cast<uint32_t*>(upoff + MH);
  const int64_t g = blockIdx.x;
  const int64_t u = a.order ? (int64_t)a.order[g] : g;
  // ---- up-hop list of the row: positives first, negatives after
  for (int k = threadIdx.x; k < a.maxhops_up; k += T)
    upraw[k] = (uint32_t)a.hop_up[(int64_t)k * a.dim_up + u];
  __syncthreads();
  if (threadIdx.x == 0) {
    int np = 0, nn = 0;
    for (int k = 0; k < a.maxhops_up; ++k) {
      const uint32_t e = upraw[k];
      const int64_t tg = (int64_t)(e & kTargetMask);
      if (tg >= a.dim_up) break;
      if (!(e & kSignBit)) upoff[np++] = tg * ld;
    }
    for (int k = 0; k < a.maxhops_up; ++k) {
      const uint32_t e = upraw[k];
      const int64_t tg = (int64_t)(e & kTargetMask);
      if (tg >= a.dim_up) break;
      if (e & kSignBit) upoff[np + nn++] = tg * ld;
    }
    npos_s = np;
    nneg_s = nn;
  }
  __syncthreads();
  const int npos = npos_s, nneg = nneg_s;
  const uint32_t ub = a.up_bits[u];
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
  const E* xrow = x + u * ld;
  for (int s = 0; s < 2; ++s) {
    const int c0 = s ? a.cstart1 : a.cstart0, c1 = s ? a.cstart2 : a.cstart1;
    const int oth = s ? a.cstart0 : a.cstart1;  // start of the other slice
    const int lds = c1 - c0;
    // ---- stage the slice through its slot map (the previous slice's gathers are done);
    // slots lds .. lds + G - 1 are zero, one in each bank group
    __syncthreads();
    for (int i = threadIdx.x; i < lds + G; i += T)
      xs[i < lds ? (i & ~(G - 1)) | a.slot_lo[c0 + i] : i] = i < lds ? xrow[c0 + i] : E(0);
    __syncthreads();
    for (int d0 = c0 + threadIdx.x * V; d0 < c1; d0 += T * V) {
      E acc[V];
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = E(0);
      // ---- down part: in-slice hops from shared memory, +1 rows first
      const uchar4 kpn = a.kpn[d0 / (32 * V)];
      const uint16_t* tp = a.dtab + d0;
      for (int k = 0; k < kpn.x; ++k) {
        const Pack<uint16_t, V> e = *reinterpret_cast<const Pack<uint16_t, V>*>(tp + (size_t)k * ld);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] += xs[e.v[v]];
      }
      for (int k = kpn.x; k < kpn.x + kpn.y; ++k) {
        const Pack<uint16_t, V> e = *reinterpret_cast<const Pack<uint16_t, V>*>(tp + (size_t)k * ld);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] -= xs[e.v[v]];
      }
      // ---- cross-slice hops from the row in global memory
      const E* xo = xrow + oth;
      const uint16_t* xp = a.xtab + d0;
      for (int k = 0; k < kpn.z; ++k) {
        const Pack<uint16_t, V> e = *reinterpret_cast<const Pack<uint16_t, V>*>(xp + (size_t)k * ld);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] += xo[e.v[v]];
      }
      for (int k = kpn.z; k < kpn.z + kpn.w; ++k) {
        const Pack<uint16_t, V> e = *reinterpret_cast<const Pack<uint16_t, V>*>(xp + (size_t)k * ld);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] -= xo[e.v[v]];
      }
      // ---- up part: the slice's columns of the neighbour rows
      const E* xb = x + d0;
#pragma unroll 8
      for (int k = 0; k < npos; ++k) {
        const Pack<E, V> q = *reinterpret_cast<const Pack<E, V>*>(xb + upoff[k]);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] += q.v[v];
      }
#pragma unroll 4
      for (int k = 0; k < nneg; ++k) {
        const Pack<E, V> q = *reinterpret_cast<const Pack<E, V>*>(xb + upoff[npos + k]);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] -= q.v[v];
      }
      // ---- diagonal and the Lanczos epilogue (as hv2_kernel)
      const Pack<uint32_t, V> db = *reinterpret_cast<const Pack<uint32_t, V>*>(a.dn_bits + d0);
      E* yp = y + u * ld + d0;
      const Pack<E, V> P = ldcs_pack(reinterpret_cast<const Pack<E, V>*>(yp));
      const Pack<uint8_t, V> lo = *reinterpret_cast<const Pack<uint8_t, V>*>(a.slot_lo + d0);
      Pack<E, V> W;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const E xc = xs[((d0 + v - c0) & ~(G - 1)) | lo.v[v]];
        const int n = __popc(ub & db.v[v]);
        if constexpr (sizeof(E) == 4) {
          const float hx = fmaf(-a.t, (float)acc[v], a.U * (float)n * (float)xc);
          const float w = fmaf(sc, hx, -bsp * (float)P.v[v]);
          W.v[v] = (E)w;
          dotf.add(w, sc * (float)xc);
        } else {
          const long long xi = (long long)xc;
          const W128 p = add128(add128(smul128(ca, (long long)acc[v]), smul128(cb, xi * n)),
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
    __syncthreads();
    if (lane == 0) {
      sm[wid][0] = (unsigned long long)doti.lo;
      sm[wid][1] = (unsigned long long)(doti.lo >> 64);
      sm[wid][2] = (unsigned long long)doti.hi;
    }
    __syncthreads();
    if (wid == 0) {
      I192 tot;
      i192_zero(tot);
      if (lane < T / 32) {
        tot.lo = ((u128)sm[lane][1] << 64) | (u128)sm[lane][0];
        tot.hi = (long long)sm[lane][2];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const I192 w = i192_shfl_down(tot, o);
        i192_add(tot, w);
      }
      if (lane == 0) {
        long long* out = reinterpret_cast<long long*>(partial) + 4 * blockIdx.x;
        out[0] = (long long)(unsigned long long)tot.lo;
        out[1] = (long long)(unsigned long long)(tot.lo >> 64);
        out[2] = tot.hi;
        out[3] = 0;
      }
    }
  }
}

}  // namespace ed

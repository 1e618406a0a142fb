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
//    of G = 128 / (R sizeof(E)) columns (G slots span all 32 banks), chosen on the host so
//    that the gathers of one request fall in distinct bank groups as far as possible; the
//    staging and epilogue accesses of a warp stay conflict-free.
//  * Down part: a per-plan table gives, for hop k of column p, the slot of the target
//    (16 bits); padding points at a zero slot. Within a chunk of 32 V columns (one warp) the
//    hops with fermion sign +1 come first and those with -1 after, each group padded to the
//    chunk's largest count, so the sign costs nothing per element; the columns are ordered
//    by (hop count, positive-hop count) to keep that padding small. Consecutive threads
//    read consecutive table entries (coalesced).
//  * Up part: each row's hop list is sorted by sign into shared memory once per CTA; the
//    threads then stream the neighbour rows with V-wide coalesced loads (L2-resident reuse).
//  * Diagonal: U popc(up[u] & dn[d]) x on the integer pipe.
// FP32 accumulates in FP32 (dot products compensated, FP64 per CTA). The int64 variant is
// the FP64-accurate path of ed_fixed.cu: exact hop sums, W = round((a S + b n X + c P) 2^k).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

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
      smem + ((size_t)(ld + 1) * sizeof(Pack<E, R>) + 15) / 16 * 16);
  uint32_t* upraw = reinterpret_cast<uint32_t*>(upoff + R * MH);
  const int64_t g0 = (int64_t)blockIdx.x * R;
  int64_t urow[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t g = g0 + r;
    urow[r] = g < a.dim_up ? (a.order ? (int64_t)a.order[g] : g) : a.dim_up;  // dim_up = none
  }

  // ---- stage the R rows (one d per thread: R coalesced loads, one vector store)
  for (int d = threadIdx.x; d <= ld; d += T) {
    Pack<E, R> p;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t u = urow[r];
      p.v[r] = (d < ld && u < a.dim_up) ? x[u * ld + d] : E(0);
    }
    xs[d < ld ? (d & ~(G - 1)) | a.slot_lo[d] : ld] = p;
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
    // at the zero slot.
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

// ------------------------------------------------------------------ host side
struct Hv2Plan {
  int kind = 0;  // 0: not usable; otherwise an index into the launch switch
  size_t smem = 0;
  int grid = 0;
  int ld = 0;
  void* dtab = nullptr;       // [rows][ld] 16-bit slots
  uchar2* kpn = nullptr;      // per chunk of 32 V columns: positive, negative table rows
  uint8_t* slot_lo = nullptr;  // per column: slot within its group of G
  uint32_t* dn_pad = nullptr;  // down bits by column
  int32_t* colpos = nullptr;  // column of each down rank
};

static int optin_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// Variants (schedule ids): R rows per CTA, V columns per thread, T threads, MB CTAs per SM
// the register allocation must allow (the occupancy the smem of small rows permits; the
// tighter bounds spill a few words).
#define HV2_KINDS(X)               \
  X(1, float, 2, 4, 256, 5)        \
  X(2, float, 1, 4, 512, 3)        \
  X(3, float, 2, 4, 256, 6)        \
  X(4, float, 1, 4, 256, 6)        \
  X(5, float, 2, 4, 512, 2)        \
  X(6, float, 4, 4, 256, 3)        \
  X(7, float, 1, 4, 512, 4)        \
  X(8, long long, 1, 2, 384, 4)    \
  X(9, long long, 1, 2, 256, 6)    \
  X(10, long long, 1, 2, 768, 2)   \
  X(11, long long, 2, 2, 512, 2)   \
  X(12, long long, 1, 2, 512, 2)   \
  X(13, long long, 2, 2, 256, 3)   \
  X(14, float, 2, 4, 256, 4)

struct KindInfo {
  size_t smem;
  int R, V, G;
  bool fx;
};

static bool kind_info(int kind, const ed_basis* b, int ld, KindInfo* ki) {
  const int MH = b->up.maxhops > 0 ? b->up.maxhops : 1;
  switch (kind) {
#define HV2_INFO(K, E, R_, V_, T, MB)                                                     \
    case K:                                                                               \
      ki->smem = ((size_t)(ld + 1) * sizeof(E) * R_ + 15) / 16 * 16 + (size_t)R_ * MH * 12; \
      ki->R = R_;                                                                         \
      ki->V = V_;                                                                         \
      ki->G = hv2_group<E, R_>();                                                         \
      ki->fx = sizeof(E) == 8;                                                            \
      return true;
    HV2_KINDS(HV2_INFO)
#undef HV2_INFO
    default:
      return false;
  }
}

// Whether variant `kind` runs this basis in this precision within the shared-memory limit.
static bool kind_usable(int kind, const ed_basis* b, bool fixed_point, int ld, KindInfo* ki) {
  if (kind <= 0 || !kind_info(kind, b, ld, ki)) return false;
  if (ki->fx != fixed_point || ki->smem > (size_t)optin_smem() || b->up.dim < ki->R) return false;
  return ld <= 0xFFFF;  // the zero slot (slot ld) must fit the 16-bit table entries
}

void hv2_free(Hv2Plan* p) {
  if (!p) return;
  if (p->dtab) cudaFree(p->dtab);
  if (p->kpn) cudaFree(p->kpn);
  if (p->slot_lo) cudaFree(p->slot_lo);
  if (p->dn_pad) cudaFree(p->dn_pad);
  if (p->colpos) cudaFree(p->colpos);
  delete p;
}

// Shared-memory slots of the staged columns. A down-gather request of the kernel is one
// hop k, one of the V columns of each lane, and a phase of G lanes (G R-element slots fill
// the 32 banks once); it costs as many wavefronts as the largest number of distinct slots
// that share a bank group (slot mod G). Slots are permuted only inside aligned groups of G
// columns, which keeps each warp's staging stores and epilogue loads conflict-free. Local
// search: take a request with a conflict, move one of its targets from the most loaded
// bank group to a free one by swapping slots with the column of its group that holds that
// free bank group; keep the swap unless the affected requests get more expensive. Fixed
// seed: the result depends only on the tables.
static std::vector<uint8_t> choose_slots(const std::vector<int32_t>& tcol, const std::vector<int>& kcount,
                                         int ld, int V, int G) {
  const int chunk = 32 * V, nch = (ld + chunk - 1) / chunk;
  std::vector<int> eoff{0}, eel;  // requests: distinct target columns (ld = zero slot)
  for (int c = 0; c < nch; ++c) {
    const int kc = kcount[c];
    for (int k = 0; k < kc; ++k)
      for (int v = 0; v < V; ++v)
        for (int p = 0; p < 32; p += G) {
          const size_t st = eel.size();
          for (int l = p; l < p + G; ++l) {
            const int q = c * chunk + l * V + v;
            if (q >= ld) continue;
            int t = tcol[(size_t)k * ld + q];
            if (t < 0) t = ld;
            if (std::find(eel.begin() + st, eel.end(), t) == eel.end()) eel.push_back(t);
          }
          if (eel.size() > st) eoff.push_back((int)eel.size());
        }
  }
  const int ne = (int)eoff.size() - 1, nn = ld + 1;
  std::vector<int> ioff((size_t)nn + 1, 0), iel;  // requests touching each column
  for (int i = 0; i < ne; ++i)
    for (int j = eoff[i]; j < eoff[i + 1]; ++j) ioff[eel[j] + 1]++;
  for (int i = 0; i < nn; ++i) ioff[i + 1] += ioff[i];
  iel.resize(ioff[nn]);
  {
    std::vector<int> fill(ioff.begin(), ioff.end() - 1);
    for (int i = 0; i < ne; ++i)
      for (int j = eoff[i]; j < eoff[i + 1]; ++j) iel[fill[eel[j]]++] = i;
  }
  std::vector<uint8_t> col((size_t)nn);
  for (int i = 0; i < nn; ++i) col[i] = (uint8_t)(i % G);
  auto cost = [&](int i) {
    uint8_t h[32] = {0};
    int m = 0;
    for (int j = eoff[i]; j < eoff[i + 1]; ++j) m = std::max(m, (int)++h[col[eel[j]]]);
    return m;
  };
  std::vector<uint8_t> ec((size_t)ne);
  for (int i = 0; i < ne; ++i) ec[i] = (uint8_t)cost(i);
  std::mt19937 rng(12345u);
  std::vector<long> mark((size_t)ne, -1);
  std::vector<int> aff;
  const long iters = ne > 0 ? 16L * ld : 0;
  for (long it = 0; it < iters; ++it) {
    const int e = (int)(rng() % (uint32_t)ne);
    if (ec[e] <= 1) continue;
    uint8_t h[32] = {0};
    int mc = 0, mx = 0;
    for (int j = eoff[e]; j < eoff[e + 1]; ++j) {
      const int x = ++h[col[eel[j]]];
      if (x > mx) mx = x, mc = col[eel[j]];
    }
    int cand[32], nc = 0, fr[32], nf = 0;
    for (int j = eoff[e]; j < eoff[e + 1]; ++j)
      if (col[eel[j]] == mc && eel[j] < ld) cand[nc++] = eel[j];
    for (int c = 0; c < G; ++c)
      if (!h[c]) fr[nf++] = c;
    if (!nc || !nf) continue;
    const int a = cand[rng() % (uint32_t)nc];
    const int tc = fr[rng() % (uint32_t)nf];
    const int base = a & ~(G - 1);
    int b = -1;
    for (int q = base; q < base + G; ++q)
      if (col[q] == tc) b = q;
    if (b < 0) continue;
    aff.clear();
    for (int j = ioff[a]; j < ioff[a + 1]; ++j)
      if (mark[iel[j]] != it) mark[iel[j]] = it, aff.push_back(iel[j]);
    for (int j = ioff[b]; j < ioff[b + 1]; ++j)
      if (mark[iel[j]] != it) mark[iel[j]] = it, aff.push_back(iel[j]);
    int before = 0, after = 0;
    for (int i : aff) before += ec[i];
    std::swap(col[a], col[b]);
    for (int i : aff) after += cost(i);
    if (after <= before) {
      for (int i : aff) ec[i] = (uint8_t)cost(i);
    } else {
      std::swap(col[a], col[b]);
    }
  }
  col.resize((size_t)ld);
  return col;
}

// Column order of the down states (by hop count, most first; ties by rank) and the tables of
// one variant, built on the host from the basis tables and uploaded.
static ed_status build_down_tables(const ed_basis* b, int ld, const KindInfo& ki, cudaStream_t s,
                                   Hv2Plan* p) {
  const int64_t n = b->dn.dim;
  const int mh = b->dn.maxhops;
  std::vector<int32_t> hop((size_t)mh * n);
  std::vector<uint32_t> bits((size_t)n);
  if (mh > 0)
    ED_TRY_CUDA(cudaMemcpyAsync(hop.data(), b->dn.hop, hop.size() * 4, cudaMemcpyDeviceToHost, s));
  ED_TRY_CUDA(cudaMemcpyAsync(bits.data(), b->dn.bits, bits.size() * 4, cudaMemcpyDeviceToHost, s));
  ED_TRY_CUDA(cudaStreamSynchronize(s));
  std::vector<int> np((size_t)n, 0), nn((size_t)n, 0);  // hops with sign +1 / -1
  for (int k = 0; k < mh; ++k)
    for (int64_t d = 0; d < n; ++d) {
      const uint32_t h = (uint32_t)hop[(size_t)k * n + d];
      if ((int64_t)(h & kTargetMask) < n) ++((h & kSignBit) ? nn : np)[d];
    }
  std::vector<int32_t> perm((size_t)n), pos((size_t)n);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t x, int32_t y) {
    const int cx = np[x] + nn[x], cy = np[y] + nn[y];
    return cx != cy ? cx > cy : np[x] > np[y];
  });
  for (int64_t q = 0; q < n; ++q) pos[perm[q]] = (int32_t)q;

  // per chunk: rows [0, kp) positive hops, [kp, kp + kn) negative hops
  const int chunk = 32 * ki.V;
  const int nchunks = (ld + chunk - 1) / chunk;
  std::vector<int> kp((size_t)nchunks, 0), kn((size_t)nchunks, 0), kcount((size_t)nchunks, 0);
  for (int64_t q = 0; q < n; ++q) {
    kp[q / chunk] = std::max(kp[q / chunk], np[perm[q]]);
    kn[q / chunk] = std::max(kn[q / chunk], nn[perm[q]]);
  }
  int rows = 1;
  for (int c = 0; c < nchunks; ++c) {
    if (kp[c] > 255 || kn[c] > 255) {
      set_error("H.v tables: more than 255 down hops of one sign");
      return ED_ERR_ARG;
    }
    kcount[c] = kp[c] + kn[c];
    rows = std::max(rows, kcount[c]);
  }
  std::vector<int32_t> tcol((size_t)rows * ld, -1);  // target column, -1 = zero slot
  for (int64_t q = 0; q < n; ++q) {
    const int c = (int)(q / chunk);
    int ip = 0, in = kp[c];
    for (int k = 0; k < mh; ++k) {
      const uint32_t h = (uint32_t)hop[(size_t)k * n + perm[q]];
      const uint32_t tg = h & kTargetMask;
      if ((int64_t)tg >= n) continue;
      const int row = (h & kSignBit) ? in++ : ip++;
      tcol[(size_t)row * ld + q] = pos[tg];
    }
  }
  const std::vector<uint8_t> lo = choose_slots(tcol, kcount, ld, ki.V, ki.G);
  std::vector<uint16_t> tab((size_t)rows * ld);
  for (size_t i = 0; i < tcol.size(); ++i) {
    const int32_t t = tcol[i];
    tab[i] = (uint16_t)(t >= 0 ? (t & ~(ki.G - 1)) | lo[t] : ld);
  }
  std::vector<uchar2> kpnv((size_t)nchunks);
  for (int c = 0; c < nchunks; ++c) kpnv[c] = make_uchar2((unsigned char)kp[c], (unsigned char)kn[c]);
  std::vector<uint32_t> pad((size_t)ld, 0u);
  for (int64_t q = 0; q < n; ++q) pad[q] = bits[perm[q]];

  if (cudaMalloc(&p->dtab, tab.size() * 2) != cudaSuccess ||
      cudaMalloc((void**)&p->kpn, kpnv.size() * sizeof(uchar2)) != cudaSuccess ||
      cudaMalloc((void**)&p->slot_lo, (size_t)ld) != cudaSuccess ||
      cudaMalloc((void**)&p->dn_pad, (size_t)ld * 4) != cudaSuccess ||
      cudaMalloc((void**)&p->colpos, (size_t)(n > 0 ? n : 1) * 4) != cudaSuccess) {
    set_error("H.v tables: out of device memory");
    return ED_ERR_OOM;
  }
  ED_TRY_CUDA(cudaMemcpyAsync(p->dtab, tab.data(), tab.size() * 2, cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaMemcpyAsync(p->kpn, kpnv.data(), kpnv.size() * sizeof(uchar2),
                              cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaMemcpyAsync(p->slot_lo, lo.data(), lo.size(), cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaMemcpyAsync(p->dn_pad, pad.data(), pad.size() * 4, cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaMemcpyAsync(p->colpos, pos.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
  return ED_OK;
}

// Choose the kernel variant for this basis and element type, build the per-plan tables.
ed_status hv2_build(const ed_basis* b, bool fixed_point, int ld, int schedule, cudaStream_t s,
                    Hv2Plan** out) {
  *out = nullptr;
  // down-loop lengths are stored in 8 bits
  if (b->dn.maxhops > 255) return ED_OK;  // caller falls back to the general kernels
  static const int pref_f32[] = {1, 4, 2, 6}, pref_fx[] = {8, 9, 12, 11};
  const int* pref = fixed_point ? pref_fx : pref_f32;
  const int npref = 4;
  int kind = 0;
  KindInfo ki{};
  for (int i = -1; i < npref && !kind; ++i) {
    const int k = i < 0 ? schedule : pref[i];
    if (kind_usable(k, b, fixed_point, ld, &ki)) kind = k;
  }
  if (!kind) return ED_OK;  // caller falls back to the general kernels
  Hv2Plan* p = new Hv2Plan();
  p->kind = kind;
  p->smem = ki.smem;
  p->ld = ld;
  p->grid = (int)((b->up.dim + ki.R - 1) / ki.R);
  ed_status r = build_down_tables(b, ld, ki, s, p);
  if (r != ED_OK) {
    hv2_free(p);
    return r;
  }
  cudaError_t e = cudaSuccess;
#define HV2_ATTR(K, E, R_, V, T, MB)                                                     \
  if (kind == K)                                                                          \
    e = cudaFuncSetAttribute(hv2_kernel<E, R_, V, T, MB>,                                 \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ki.smem);
  HV2_KINDS(HV2_ATTR)
#undef HV2_ATTR
  if (e != cudaSuccess) {
    hv2_free(p);
    set_error("H.v tables: %s", cudaGetErrorString(e));
    return ED_ERR_CUDA;
  }
  *out = p;
  return ED_OK;
}

const int32_t* hv2_colpos(const Hv2Plan* p) { return p ? p->colpos : nullptr; }

int hv2_grid(const Hv2Plan* p) { return p ? p->grid : 0; }

ed_status hv2_autotune(const ed_basis* b, bool fixed_point, int ld, void* x, void* y,
                       const LzScalars* S, void* partial, cudaStream_t s, int* kind) {
  *kind = 0;
  static const int cand_f32[] = {1, 2, 3, 4, 5, 6, 7, 14}, cand_fx[] = {8, 9, 10, 11, 12, 13};
  const int* cand = fixed_point ? cand_fx : cand_f32;
  const int nc = fixed_point ? 6 : 8;
  constexpr int kReps = 5;
  cudaEvent_t ev[kReps + 1];
  for (auto& e : ev) ED_TRY_CUDA(cudaEventCreate(&e));
  float best = 1e30f;
  ed_status r = ED_OK;
  for (int i = 0; i < nc && r == ED_OK; ++i) {
    KindInfo ki;
    if (!kind_usable(cand[i], b, fixed_point, ld, &ki)) continue;
    Hv2Plan* p = nullptr;
    if ((r = hv2_build(b, fixed_point, ld, cand[i], s, &p)) != ED_OK) break;
    if (!p || p->kind != cand[i]) {
      hv2_free(p);
      continue;
    }
    // two warm-up launches, then the median of kReps individually timed launches
    for (int k = 0; k < 2 && r == ED_OK; ++k) r = hv2_launch(p, b, 1.0, 1.0, x, y, S, 0, partial, s);
    float ms = 0.f;
    if (r == ED_OK) {
      cudaEventRecord(ev[0], s);
      for (int k = 0; k < kReps && r == ED_OK; ++k) {
        r = hv2_launch(p, b, 1.0, 1.0, x, y, S, 0, partial, s);
        cudaEventRecord(ev[k + 1], s);
      }
      float t[kReps];
      if (r == ED_OK && cudaEventSynchronize(ev[kReps]) == cudaSuccess) {
        for (int k = 0; k < kReps; ++k) cudaEventElapsedTime(&t[k], ev[k], ev[k + 1]);
        std::sort(t, t + kReps);
        ms = t[kReps / 2];
      } else if (r == ED_OK) {
        set_error("H.v autotune: timing failed");
        r = ED_ERR_CUDA;
      }
    }
    hv2_free(p);
    if (r == ED_OK && ms < best) best = ms, *kind = cand[i];
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return r;
}
int hv2_kind(const Hv2Plan* p) { return p ? p->kind : 0; }

ed_status hv2_launch(const Hv2Plan* p, const ed_basis* b, double t, double U, const void* x,
                     void* y, const LzScalars* S, int cur, void* partial, cudaStream_t s) {
  Hv2Args a;
  a.up_bits = b->up.bits;
  a.dn_bits = p->dn_pad;
  a.dtab = (const uint16_t*)p->dtab;
  a.kpn = p->kpn;
  a.slot_lo = p->slot_lo;
  a.hop_up = b->up.hop;
  a.order = b->up_order;
  a.dim_up = b->up.dim;
  a.ld = p->ld;
  a.maxhops_up = b->up.maxhops;
  a.t = (float)t;
  a.U = (float)U;
#define HV2_LAUNCH(K, E, R_, V, T, MB)                                                     \
  if (p->kind == K)                                                                         \
    hv2_kernel<E, R_, V, T, MB><<<p->grid, T, p->smem, s>>>(a, (const E*)x, (E*)y, S, cur, \
                                                             partial);
  HV2_KINDS(HV2_LAUNCH)
#undef HV2_LAUNCH
  ED_TRY_CUDA(cudaGetLastError());
  return ED_OK;
}

}  // namespace ed

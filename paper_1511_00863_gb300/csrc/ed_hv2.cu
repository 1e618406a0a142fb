// Host side of the Lanczos-fused H.v (kernel in ed_hv2_kernel.cuh): the variant table, the
// per-plan down tables (column order by hop count and sign, shared-memory slot map), the
// autotuner and the launch.
#include <algorithm>
#include <cstring>
#include <deque>
#include <mutex>
#include <numeric>
#include <random>
#include <vector>

#include "ed_hv2_kernel.cuh"
#include "ed_hv2c_kernel.cuh"

namespace ed {

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

// Complex FP32 variants (ED_C32; hv2c_kernel): id, R, V, T, MB.
#define HV2C_KINDS(X)        \
  X(20, 2, 2, 256, 4)        \
  X(21, 1, 2, 256, 6)        \
  X(22, 1, 2, 512, 3)        \
  X(23, 2, 2, 512, 2)

struct KindInfo {
  size_t smem;
  int R, V, G;
  int mode;  // kHv2F32, kHv2Fx, kHv2C32
};

// Entries of the signed amplitude table of the complex kernel.
static int hv2c_namp(const ed_basis* b) { return b->has_tau() ? 4 * b->n_bonds : 2; }

static bool kind_info(int kind, const ed_basis* b, int ld, KindInfo* ki) {
  const int MH = b->up.maxhops > 0 ? b->up.maxhops : 1;
  switch (kind) {
#define HV2_INFO(K, E, R_, V_, T, MB)                                                     \
    case K:                                                                               \
      ki->smem = ((size_t)(ld + hv2_group<E, R_>()) * sizeof(E) * R_ + 15) / 16 * 16 +      \
                 (size_t)R_ * MH * 12;                                                    \
      ki->R = R_;                                                                         \
      ki->V = V_;                                                                         \
      ki->G = hv2_group<E, R_>();                                                         \
      ki->mode = sizeof(E) == 8 ? kHv2Fx : kHv2F32;                                       \
      return true;
    HV2_KINDS(HV2_INFO)
#undef HV2_INFO
#define HV2C_INFO(K, R_, V_, T, MB)                                                         \
    case K:                                                                                 \
      ki->smem = (size_t)(ld + hv2_group<float2, R_>()) * 8 * R_ +                          \
                 (size_t)((hv2c_namp(b) + 1) & ~1) * 8 + (size_t)R_ * MH * 12;              \
      ki->R = R_;                                                                           \
      ki->V = V_;                                                                           \
      ki->G = hv2_group<float2, R_>();                                                      \
      ki->mode = kHv2C32;                                                                   \
      return true;
    HV2C_KINDS(HV2C_INFO)
#undef HV2C_INFO
    default:
      return false;
  }
}

// Whether variant `kind` runs this basis in this precision within the shared-memory limit.
static bool kind_usable(int kind, const ed_basis* b, int mode, int ld, KindInfo* ki) {
  if (kind <= 0 || !kind_info(kind, b, ld, ki)) return false;
  if (ki->mode != mode || ki->smem > (size_t)optin_smem() || b->up.dim < ki->R) return false;
  if (mode == kHv2C32 && hv2c_namp(b) > 0x10000) return false;  // 16-bit amplitude index
  return ld + ki->G - 1 <= 0xFFFF;  // the zero slots must fit the 16-bit slot field
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

// Down-gather groups. One warp-wide gather of the kernel (hop step k, one of the V columns
// of each lane) is served in phases of G lanes (G R-element slots fill the 32 banks once);
// a phase costs as many shared-memory wavefronts as the largest number of distinct slots
// in one bank group (slot mod G). A group is one chunk, one sign (table rows [k0, k0 + K):
// the positive hops, then the negative ones; one group of all hops for the complex kernel),
// one column v of the lanes and one phase: G columns whose hops run in the same K steps.
struct GatherGroup {
  int c, v, p;  // chunk, column within the lane, first lane of the phase
  int k0, K;    // table rows
};

static std::vector<GatherGroup> gather_groups(int ld, int V, int G, const std::vector<int>& kp,
                                              const std::vector<int>& kn) {
  std::vector<GatherGroup> gg;
  const int nch = (int)kp.size();
  for (int c = 0; c < nch; ++c)
    for (int sg = 0; sg < 2; ++sg) {
      const int k0 = sg ? kp[c] : 0, K = sg ? kn[c] : kp[c];
      if (K == 0) continue;
      for (int v = 0; v < V; ++v)
        for (int p = 0; p < 32; p += G)
          if (c * 32 * V + p * V + v < ld) gg.push_back({c, v, p, k0, K});
    }
  return gg;
}

static inline int group_column(const GatherGroup& g, int l, int V) {
  return g.c * 32 * V + (g.p + l) * V + g.v;
}

// Slot map: lo[p] for every column, a permutation inside each aligned group of G columns
// (so slot mod G = lo[p]). The hops of a group can be reordered per lane (below), so what
// matters is how many of the group's hops land in each bank group: at most K each allows a
// conflict-free order (a bipartite graph of maximum degree K has a K-edge-colouring). The
// search lowers the excess over K, summed over bank groups and groups (squares as the tie
// break): take a group with an over-full and an under-full bank group, move one target of
// the first to the second by swapping lo with the column of its aligned group that holds
// it, keep the swap unless the affected groups get worse. Fixed seed: the result depends
// only on the tables.
static std::vector<uint8_t> choose_slots(const std::vector<int32_t>& tcol,
                                         const std::vector<GatherGroup>& gg, int ld, int V,
                                         int G) {
  const int ng = (int)gg.size();
  std::vector<int> goff{0}, gcol, gcnt, tmp;  // per group: distinct targets and multiplicity
  for (const GatherGroup& g : gg) {
    tmp.clear();
    for (int l = 0; l < G; ++l) {
      const int q = group_column(g, l, V);
      if (q >= ld) continue;
      for (int k = 0; k < g.K; ++k) {
        const int t = tcol[(size_t)(g.k0 + k) * ld + q];
        if (t >= 0) tmp.push_back(t);
      }
    }
    std::sort(tmp.begin(), tmp.end());
    for (size_t i = 0; i < tmp.size();) {
      size_t j = i;
      while (j < tmp.size() && tmp[j] == tmp[i]) ++j;
      gcol.push_back(tmp[i]);
      gcnt.push_back((int)(j - i));
      i = j;
    }
    goff.push_back((int)gcol.size());
  }
  std::vector<int> ooff((size_t)ld + 1, 0), ogrp, ocnt;  // groups that gather each column
  for (int x : gcol) ++ooff[x + 1];
  for (int i = 0; i < ld; ++i) ooff[i + 1] += ooff[i];
  ogrp.resize(gcol.size());
  ocnt.resize(gcol.size());
  {
    std::vector<int> fill(ooff.begin(), ooff.end() - 1);
    for (int g = 0; g < ng; ++g)
      for (int j = goff[g]; j < goff[g + 1]; ++j) {
        ogrp[fill[gcol[j]]] = g;
        ocnt[fill[gcol[j]]++] = gcnt[j];
      }
  }
  std::vector<uint8_t> col((size_t)ld);
  for (int i = 0; i < ld; ++i) col[i] = (uint8_t)(i % G);
  std::vector<int> h((size_t)ng * G, 0);  // hops of each group per bank group
  for (int g = 0; g < ng; ++g)
    for (int j = goff[g]; j < goff[g + 1]; ++j) h[(size_t)g * G + col[gcol[j]]] += gcnt[j];
  auto f = [](long e) { return e > 0 ? 1024 * e + e * e : 0L; };  // cost of an excess e
  // a swap changes only bank groups co and cu of the groups gathering a or b
  auto pair_cost = [&](int g, int co, int cu) {
    return f(h[(size_t)g * G + co] - gg[g].K) + f(h[(size_t)g * G + cu] - gg[g].K);
  };
  std::mt19937 rng(12345u);
  std::vector<long> mark((size_t)ng, -1);
  std::vector<int> aff;
  const long iters = ng > 0 ? 48L * ld : 0;
  for (long it = 0; it < iters; ++it) {
    const int g = (int)(rng() % (uint32_t)ng);
    const int nt = goff[g + 1] - goff[g];
    if (nt == 0) continue;
    const int a = gcol[goff[g] + (int)(rng() % (uint32_t)nt)];
    const int co = col[a];
    const int* hg = &h[(size_t)g * G];
    if (hg[co] <= gg[g].K) continue;
    int under[32], nu = 0;
    for (int b = 0; b < G; ++b)
      if (hg[b] < gg[g].K) under[nu++] = b;
    if (!nu) continue;
    const int cu = under[rng() % (uint32_t)nu];
    int b = -1;
    for (int q = a & ~(G - 1); q < (a & ~(G - 1)) + G; ++q)
      if (col[q] == cu) b = q;
    if (b < 0) continue;
    aff.clear();
    for (int j = ooff[a]; j < ooff[a + 1]; ++j)
      if (mark[ogrp[j]] != it) mark[ogrp[j]] = it, aff.push_back(ogrp[j]);
    for (int j = ooff[b]; j < ooff[b + 1]; ++j)
      if (mark[ogrp[j]] != it) mark[ogrp[j]] = it, aff.push_back(ogrp[j]);
    long before = 0, after = 0;
    for (int x : aff) before += pair_cost(x, co, cu);
    auto move = [&](int from, int to) {
      for (int j = ooff[a]; j < ooff[a + 1]; ++j) {
        h[(size_t)ogrp[j] * G + from] -= ocnt[j];
        h[(size_t)ogrp[j] * G + to] += ocnt[j];
      }
      for (int j = ooff[b]; j < ooff[b + 1]; ++j) {
        h[(size_t)ogrp[j] * G + to] -= ocnt[j];
        h[(size_t)ogrp[j] * G + from] += ocnt[j];
      }
    };
    move(co, cu);
    for (int x : aff) after += pair_cost(x, co, cu);
    if (after <= before) {
      std::swap(col[a], col[b]);
    } else {
      move(cu, co);
    }
  }
  return col;
}

// Hop order inside each group: the hops of the G lanes are the edges of a bipartite graph
// between lanes and bank groups, and the K steps colour its edges, so that no lane takes
// two hops in one step. Each bank group is split into nodes of at most K hops, so every
// node has degree <= K and a K-edge-colouring exists (Koenig); it is built edge by edge,
// swapping two colours along an alternating path where the free ones differ. A step then
// meets a bank group as often as that group has nodes used in it: once when its hops fit.
// Padding entries become the zero slot (ld + bank group) of a bank group the step leaves
// free. Rows of tcol (and the amplitude indices `tamp`, when given) are permuted within
// each group's rows; a zero slot is stored as ld + bank group.
static void schedule_gathers(std::vector<int32_t>& tcol, std::vector<uint32_t>& tamp,
                             const std::vector<GatherGroup>& gg, const std::vector<uint8_t>& lo,
                             int ld, int V, int G) {
  std::vector<int> eu, ew, erow, ec, at, path, base, deg;
  std::vector<int32_t> old_t;
  std::vector<uint32_t> old_a;
  std::vector<uint32_t> used;
  for (const GatherGroup& g : gg) {
    const int K = g.K;
    deg.assign((size_t)G, 0);
    for (int l = 0; l < G; ++l) {
      const int q = group_column(g, l, V);
      if (q >= ld) continue;
      for (int k = 0; k < K; ++k) {
        const int t = tcol[(size_t)(g.k0 + k) * ld + q];
        if (t >= 0) ++deg[lo[t]];
      }
    }
    base.assign((size_t)G + 1, G);  // node ids: lanes [0, G), then the bank-group nodes
    for (int b = 0; b < G; ++b) base[b + 1] = base[b] + (deg[b] + K - 1) / K;
    const int nnodes = base[G];
    eu.clear(), ew.clear(), erow.clear();
    std::vector<int> seen((size_t)G, 0);
    for (int l = 0; l < G; ++l) {
      const int q = group_column(g, l, V);
      if (q >= ld) continue;
      for (int k = 0; k < K; ++k) {
        const int t = tcol[(size_t)(g.k0 + k) * ld + q];
        if (t < 0) continue;
        const int b = lo[t];
        eu.push_back(l);
        ew.push_back(base[b] + seen[b]++ / K);
        erow.push_back(k);
      }
    }
    const int E = (int)eu.size();
    ec.assign((size_t)E, -1);
    at.assign((size_t)nnodes * K, -1);
    bool ok = true;
    for (int e = 0; e < E && ok; ++e) {
      const int u = eu[e], w = ew[e];
      int a = -1, b = -1;
      for (int s = 0; s < K && a < 0; ++s)
        if (at[(size_t)u * K + s] < 0) a = s;
      for (int s = 0; s < K && b < 0; ++s)
        if (at[(size_t)w * K + s] < 0) b = s;
      if (a < 0 || b < 0) {
        ok = false;
        break;
      }
      if (at[(size_t)w * K + a] >= 0) {  // swap colours a and b along the path from w
        path.clear();
        int node = w, want = a;
        for (int pe; (pe = at[(size_t)node * K + want]) >= 0;) {
          path.push_back(pe);
          if ((int)path.size() > E) {
            ok = false;
            break;
          }
          node = eu[pe] == node ? ew[pe] : eu[pe];
          want = want == a ? b : a;
        }
        if (!ok) break;
        for (int pe : path) at[(size_t)eu[pe] * K + ec[pe]] = at[(size_t)ew[pe] * K + ec[pe]] = -1;
        for (int pe : path) {
          ec[pe] = ec[pe] == a ? b : a;
          at[(size_t)eu[pe] * K + ec[pe]] = at[(size_t)ew[pe] * K + ec[pe]] = pe;
        }
      }
      ec[e] = a;
      at[(size_t)u * K + a] = at[(size_t)w * K + a] = e;
    }
    if (!ok) ec.assign((size_t)E, -1);  // cannot happen; keep the original order
    used.assign((size_t)K, 0u);
    for (int e = 0; e < E; ++e) {
      const int s = ec[e] >= 0 ? ec[e] : erow[e];
      const int q = group_column(g, eu[e], V);
      used[s] |= 1u << lo[tcol[(size_t)(g.k0 + erow[e]) * ld + q]];
    }
    // write the lanes back in their new order, padding on a free zero slot
    for (int l = 0, e = 0; l < G; ++l) {
      const int q = group_column(g, l, V);
      if (q >= ld) continue;
      old_t.resize((size_t)K);
      old_a.resize((size_t)K);
      for (int k = 0; k < K; ++k) {
        old_t[k] = tcol[(size_t)(g.k0 + k) * ld + q];
        if (!tamp.empty()) old_a[k] = tamp[(size_t)(g.k0 + k) * ld + q];
        tcol[(size_t)(g.k0 + k) * ld + q] = -1;
      }
      for (; e < E && eu[e] == l; ++e) {
        const int s = ec[e] >= 0 ? ec[e] : erow[e];
        tcol[(size_t)(g.k0 + s) * ld + q] = old_t[erow[e]];
        if (!tamp.empty()) tamp[(size_t)(g.k0 + s) * ld + q] = old_a[erow[e]];
      }
      for (int k = 0; k < K; ++k) {
        int32_t& t = tcol[(size_t)(g.k0 + k) * ld + q];
        if (t >= 0) continue;
        const uint32_t freeb = ~used[k] & (G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u));
        t = ld + (freeb ? __builtin_ctz(freeb) : 0);
        if (!tamp.empty()) tamp[(size_t)(g.k0 + k) * ld + q] = 0u;
      }
    }
  }
}

// Down-state column order and per-geometry tables, built on the host from the basis tables:
// columns ordered by hop count (most first), then by +1-hop count, then by rank; per chunk of
// 32 V columns the table rows [0, kp) hold the +1 hops and [kp, kp + kn) the -1 hops as
// shared-memory slots, each column's hops in the order schedule_gathers gives them.
// Variants with the same (V, G) share them; the basis caches them.
struct DownTables {
  int V = 0, G = 0, ld = 0;
  bool cplx = false;              // complex kernel: 32-bit entries slot | amplitude index << 16
  std::vector<uint16_t> tab;
  std::vector<uint32_t> tab32;
  std::vector<uchar2> kpn;
  std::vector<uint8_t> lo;
  std::vector<uint32_t> pad;
  std::vector<int32_t> pos;
};
static std::mutex g_tables_mu;

// Column order of the down states (by hop count, most first; ties by rank) and the tables of
// one variant, built on the host from the basis tables and uploaded.
static ed_status compute_down_tables(const ed_basis* b, int ld, const KindInfo& ki, cudaStream_t s,
                                     DownTables& out) {
  const int64_t n = b->dn.dim;
  const int mh = b->dn.maxhops;
  const bool cplx = ki.mode == kHv2C32;
  std::vector<int32_t> hop((size_t)mh * n), hopa;
  std::vector<uint32_t> bits((size_t)n);
  if (mh > 0)
    ED_TRY_CUDA(cudaMemcpyAsync(hop.data(), b->dn.hop, hop.size() * 4, cudaMemcpyDeviceToHost, s));
  if (cplx && mh > 0 && b->dn.hopa) {
    hopa.resize(hop.size());
    ED_TRY_CUDA(cudaMemcpyAsync(hopa.data(), b->dn.hopa, hopa.size() * 4, cudaMemcpyDeviceToHost, s));
  }
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
    if (cplx) {  // one loop over all hops: the sign is in the amplitude
      kp[q / chunk] = std::max(kp[q / chunk], np[perm[q]] + nn[perm[q]]);
    } else {
      kp[q / chunk] = std::max(kp[q / chunk], np[perm[q]]);
      kn[q / chunk] = std::max(kn[q / chunk], nn[perm[q]]);
    }
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
  std::vector<uint32_t> tamp(cplx ? tcol.size() : 0, 0u);  // signed amplitude index
  for (int64_t q = 0; q < n; ++q) {
    const int c = (int)(q / chunk);
    int ip = 0, in = kp[c];
    for (int k = 0; k < mh; ++k) {
      const uint32_t h = (uint32_t)hop[(size_t)k * n + perm[q]];
      const uint32_t tg = h & kTargetMask;
      if ((int64_t)tg >= n) continue;
      const int row = cplx ? ip++ : (h & kSignBit) ? in++ : ip++;
      tcol[(size_t)row * ld + q] = pos[tg];
      if (cplx) {
        const uint32_t num = hopa.empty() ? 0u : (uint32_t)hopa[(size_t)k * n + perm[q]];
        tamp[(size_t)row * ld + q] = 2u * num + (h >> 31);
      }
    }
  }
  const std::vector<GatherGroup> gg = gather_groups(ld, ki.V, ki.G, kp, kn);
  out.lo = choose_slots(tcol, gg, ld, ki.V, ki.G);
  const std::vector<uint8_t>& lo = out.lo;
  schedule_gathers(tcol, tamp, gg, lo, ld, ki.V, ki.G);
  // slot of a table entry: the target's, a zero slot as stored, or the first zero slot
  auto slot = [&](int32_t t) {
    return (uint32_t)(t < 0 ? ld : t >= ld ? t : (t & ~(ki.G - 1)) | lo[t]);
  };
  out.cplx = cplx;
  if (cplx) {
    out.tab32.assign((size_t)rows * ld, 0u);
    for (size_t i = 0; i < tcol.size(); ++i) out.tab32[i] = slot(tcol[i]) | (tamp[i] << 16);
  } else {
    std::vector<uint16_t>& tab = out.tab;
    tab.assign((size_t)rows * ld, 0);
    for (size_t i = 0; i < tcol.size(); ++i) tab[i] = (uint16_t)slot(tcol[i]);
  }
  std::vector<uchar2>& kpnv = out.kpn;
  kpnv.resize((size_t)nchunks);
  for (int c = 0; c < nchunks; ++c) kpnv[c] = make_uchar2((unsigned char)kp[c], (unsigned char)kn[c]);
  out.pad.assign((size_t)ld, 0u);
  for (int64_t q = 0; q < n; ++q) out.pad[q] = bits[perm[q]];
  out.pos = pos;
  out.V = ki.V;
  out.G = ki.G;
  out.ld = ld;
  return ED_OK;
}

static ed_status upload_down_tables(const DownTables& t, int64_t n, cudaStream_t s, Hv2Plan* p) {
  const int ld = t.ld;
  const size_t tbytes = t.cplx ? t.tab32.size() * 4 : t.tab.size() * 2;
  const void* tdata = t.cplx ? (const void*)t.tab32.data() : (const void*)t.tab.data();
  if (cudaMalloc(&p->dtab, tbytes) != cudaSuccess ||
      cudaMalloc((void**)&p->kpn, t.kpn.size() * sizeof(uchar2)) != cudaSuccess ||
      cudaMalloc((void**)&p->slot_lo, (size_t)ld) != cudaSuccess ||
      cudaMalloc((void**)&p->dn_pad, (size_t)ld * 4) != cudaSuccess ||
      cudaMalloc((void**)&p->colpos, (size_t)(n > 0 ? n : 1) * 4) != cudaSuccess) {
    set_error("H.v tables: out of device memory");
    return ED_ERR_OOM;
  }
  ED_TRY_CUDA(cudaMemcpyAsync(p->dtab, tdata, tbytes, cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaMemcpyAsync(p->kpn, t.kpn.data(), t.kpn.size() * sizeof(uchar2),
                              cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaMemcpyAsync(p->slot_lo, t.lo.data(), t.lo.size(), cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaMemcpyAsync(p->dn_pad, t.pad.data(), t.pad.size() * 4, cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaMemcpyAsync(p->colpos, t.pos.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaStreamSynchronize(s));
  return ED_OK;
}


// The cached tables of this geometry, computed on first use.
static ed_status down_tables(const ed_basis* b, int ld, const KindInfo& ki, cudaStream_t s,
                             const DownTables** out) {
  std::lock_guard<std::mutex> lock(g_tables_mu);
  auto* cache = static_cast<std::deque<DownTables>*>(b->hv2_tables);
  if (!cache) b->hv2_tables = cache = new std::deque<DownTables>();
  for (const DownTables& t : *cache)
    if (t.V == ki.V && t.G == ki.G && t.ld == ld && t.cplx == (ki.mode == kHv2C32)) {
      *out = &t;
      return ED_OK;
    }
  DownTables t;
  const ed_status r = compute_down_tables(b, ld, ki, s, t);
  if (r != ED_OK) return r;
  cache->push_back(std::move(t));
  *out = &cache->back();  // a deque keeps its elements in place as it grows
  return ED_OK;
}

void hv2_tables_free(const ed_basis* b) {
  std::lock_guard<std::mutex> lock(g_tables_mu);
  delete static_cast<std::deque<DownTables>*>(b->hv2_tables);
  b->hv2_tables = nullptr;
}

// Choose the kernel variant for this basis and element type, build the per-plan tables.
ed_status hv2_build(const ed_basis* b, int mode, int ld, int schedule, cudaStream_t s,
                    Hv2Plan** out) {
  *out = nullptr;
  // down-loop lengths are stored in 8 bits
  if (b->dn.maxhops > 255) return ED_OK;  // caller falls back to the general kernels
  static const int pref_f32[] = {1, 4, 2, 6}, pref_fx[] = {8, 9, 12, 11}, pref_c32[] = {20, 21, 22, 23};
  const int* pref = mode == kHv2Fx ? pref_fx : mode == kHv2C32 ? pref_c32 : pref_f32;
  const int npref = 4;
  int kind = 0;
  KindInfo ki{};
  for (int i = -1; i < npref && !kind; ++i) {
    const int k = i < 0 ? schedule : pref[i];
    if (i >= 0 && b->up.dim < kMinRowsStaged) break;  // few rows: the general kernels
    if (kind_usable(k, b, mode, ld, &ki)) kind = k;
  }
  if (!kind) return ED_OK;  // caller falls back to the general kernels
  Hv2Plan* p = new Hv2Plan();
  p->kind = kind;
  p->smem = ki.smem;
  p->ld = ld;
  p->grid = (int)((b->up.dim + ki.R - 1) / ki.R);
  const DownTables* t = nullptr;
  ed_status r = down_tables(b, ld, ki, s, &t);
  if (r == ED_OK) r = upload_down_tables(*t, b->dn.dim, s, p);
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
#define HV2C_ATTR(K, R_, V, T, MB)                                                         \
  if (kind == K)                                                                          \
    e = cudaFuncSetAttribute(hv2c_kernel<R_, V, T, MB>,                                   \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ki.smem);
  HV2C_KINDS(HV2C_ATTR)
#undef HV2C_ATTR
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

ed_status hv2_autotune(const ed_basis* b, int mode, int ld, void* x, void* y,
                       const LzScalars* S, void* partial, cudaStream_t s, int* kind) {
  *kind = 0;
  if (b->up.dim < kMinRowsStaged) return ED_OK;  // few rows: the general kernels
  static const int cand_f32[] = {1, 2, 3, 4, 5, 6, 7, 14}, cand_fx[] = {8, 9, 10, 11, 12, 13},
                   cand_c32[] = {20, 21, 22, 23};
  const int* cand = mode == kHv2Fx ? cand_fx : mode == kHv2C32 ? cand_c32 : cand_f32;
  const int nc = mode == kHv2Fx ? 6 : mode == kHv2C32 ? 4 : 8;
  constexpr int kReps = 5;
  cudaEvent_t ev[kReps + 1];
  for (auto& e : ev) ED_TRY_CUDA(cudaEventCreate(&e));
  float best = 1e30f;
  ed_status r = ED_OK;
  for (int i = 0; i < nc && r == ED_OK; ++i) {
    KindInfo ki;
    if (!kind_usable(cand[i], b, mode, ld, &ki)) continue;
    Hv2Plan* p = nullptr;
    if ((r = hv2_build(b, mode, ld, cand[i], s, &p)) != ED_OK) break;
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
  if (p->kind >= 20) {
    Hv2cArgs c;
    c.up_bits = b->up.bits;
    c.dn_bits = p->dn_pad;
    c.dtab = (const uint32_t*)p->dtab;
    c.kpn = p->kpn;
    c.slot_lo = p->slot_lo;
    c.hop_up = b->up.hop;
    c.hopa_up = b->up.hopa;
    c.order = b->up_order;
    c.tau = b->tau;
    c.dim_up = b->up.dim;
    c.ld = p->ld;
    c.maxhops_up = b->up.maxhops;
    c.namp = hv2c_namp(b);
    c.t = (float)t;
    c.U = (float)U;
#define HV2C_LAUNCH(K, R_, V, T, MB)                                                          \
    if (p->kind == K)                                                                          \
      hv2c_kernel<R_, V, T, MB><<<p->grid, T, p->smem, s>>>(c, (const float2*)x, (float2*)y, S, \
                                                             cur, (double*)partial);
    HV2C_KINDS(HV2C_LAUNCH)
#undef HV2C_LAUNCH
  }
  ED_TRY_CUDA(cudaGetLastError());
  return ED_OK;
}

}  // namespace ed

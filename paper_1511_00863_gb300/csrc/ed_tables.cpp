// Host-side plan tables of the fused H.v: column order, slot map and the per-lane order of
// the down hops (declarations and layout in ed_tables.h). Plain C++: the library builds
// them from its device tables for every plan, and ed_hv_down_tables exposes the same code
// on host arrays.
#include "ed_tables.h"

#include <algorithm>
#include <numeric>
#include <random>

namespace ed {

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

ed_status build_down_tables(const int32_t* hop, const int32_t* hopa, const uint32_t* bits,
                            int64_t n, int mh, int ld, int V, int G, bool cplx, DownTables& out) {
  if (n < 1 || mh < 0 || ld < (int)((n + 31) / 32 * 32) || ld % 32 != 0 || ld + G - 1 > 0xFFFF ||
      !(G == 8 || G == 16 || G == 32) || V < 1 || V > 8 || (mh > 0 && !hop) || !bits) {
    set_error("H.v tables: invalid geometry (n %lld, maxhops %d, ld %d, V %d, G %d)",
              (long long)n, mh, ld, V, G);
    return ED_ERR_ARG;
  }
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
  const int chunk = 32 * V;
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
        const int32_t num = hopa ? hopa[(size_t)k * n + perm[q]] : 0;
        if (num < 0 || 2 * (int64_t)num + 1 > 0xFFFF) {  // the index field has 16 bits
          set_error("H.v tables: amplitude number %d out of range", num);
          return ED_ERR_ARG;
        }
        tamp[(size_t)row * ld + q] = 2u * (uint32_t)num + (h >> 31);
      }
    }
  }
  const std::vector<GatherGroup> gg = gather_groups(ld, V, G, kp, kn);
  out.lo = choose_slots(tcol, gg, ld, V, G);
  const std::vector<uint8_t>& lo = out.lo;
  schedule_gathers(tcol, tamp, gg, lo, ld, V, G);
  // slot of a table entry: the target's, a zero slot as stored, or the first zero slot
  auto slot = [&](int32_t t) {
    return (uint32_t)(t < 0 ? ld : t >= ld ? t : (t & ~(G - 1)) | lo[t]);
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
  out.kpn.resize(2 * (size_t)nchunks);
  for (int c = 0; c < nchunks; ++c) {
    out.kpn[2 * c] = (uint8_t)kp[c];
    out.kpn[2 * c + 1] = (uint8_t)kn[c];
  }
  out.pad.assign((size_t)ld, 0u);
  for (int64_t q = 0; q < n; ++q) out.pad[q] = bits[perm[q]];
  out.pos = pos;
  out.V = V;
  out.G = G;
  out.ld = ld;
  out.rows = rows;
  return ED_OK;
}

}  // namespace ed

extern "C" ed_status ed_hv_down_tables(const int32_t* hop, const int32_t* hop_amp,
                                       const uint32_t* bits, int64_t dim, int32_t maxhops,
                                       int32_t ld, int32_t V, int32_t G, int32_t complex_entries,
                                       uint32_t* table, int32_t rows_cap, int32_t* rows,
                                       uint8_t* kpn, uint8_t* slot_lo, int32_t* colpos) {
  if (!table || !rows || !kpn || !slot_lo || !colpos || rows_cap < 0) {
    ed::set_error("ed_hv_down_tables: null output or negative rows_cap");
    return ED_ERR_ARG;
  }
  ed::DownTables t;
  const ed_status r = ed::build_down_tables(hop, hop_amp, bits, dim, maxhops, ld, V, G,
                                            complex_entries != 0, t);
  if (r != ED_OK) return r;
  *rows = t.rows;
  if (t.rows > rows_cap) {
    ed::set_error("ed_hv_down_tables: %d table rows needed, rows_cap %d", t.rows, rows_cap);
    return ED_ERR_ARG;
  }
  const size_t ne = (size_t)t.rows * (size_t)ld;
  for (size_t i = 0; i < ne; ++i) table[i] = t.cplx ? t.tab32[i] : (uint32_t)t.tab[i];
  std::copy(t.kpn.begin(), t.kpn.end(), kpn);
  std::copy(t.lo.begin(), t.lo.end(), slot_lo);
  std::copy(t.pos.begin(), t.pos.end(), colpos);
  return ED_OK;
}

namespace ed {

// Split-row tables: the down states are cut in two slices by the occupation of one site
// (slice 0: occupied, slice 1: empty); a slice is staged in shared memory at a time, so a
// row twice as long as shared memory can still be processed row-staged. Each slice gets the
// plain tables of its own states (build_down_tables on the slice's sub-basis with the hops
// that stay inside it: column order, slot map, per-lane hop order against bank conflicts,
// zero slots ld_s .. ld_s + G - 1); slice s occupies the columns [cstart[s], cstart[s+1]),
// ld_s = cstart[s+1] - cstart[s] a multiple of 32 V with at least one padding column. The
// hops into the other slice go to rows of their own (xtab: the target's column inside the
// other slice, read from global memory; padding points at the other slice's last column,
// a padding column that holds 0). Per chunk of 32 V columns kpn holds four counts: in-slice
// +1 rows, in-slice -1 rows, cross +1 rows, cross -1 rows.
ed_status build_split_tables(const int32_t* hop, const uint32_t* bits, int64_t n, int mh, int V,
                             int G, int site, SplitTables& out) {
  if (n < 1 || mh < 0 || V < 1 || V > 8 || site < 0 || site > 31 || !(G == 8 || G == 16 || G == 32)) {
    set_error("split tables: invalid geometry");
    return ED_ERR_ARG;
  }
  const int CW = 32 * V;
  std::vector<int64_t> members[2];
  std::vector<int> slice((size_t)n), local((size_t)n);
  for (int64_t d = 0; d < n; ++d) {
    const int sl = ((bits[d] >> site) & 1u) ? 0 : 1;
    slice[d] = sl;
    local[d] = (int)members[sl].size();
    members[sl].push_back(d);
  }
  out = SplitTables();
  out.V = V;
  out.G = G;
  out.site = site;
  int lds[2];
  for (int sl = 0; sl < 2; ++sl) {
    const int64_t ns = (int64_t)members[sl].size();
    lds[sl] = (int)((ns + 1 + CW - 1) / CW * CW);  // at least one padding column
  }
  if (lds[0] + G > 65536 || lds[1] + G > 65536) {  // slots and columns are 16-bit entries
    set_error("split tables: a slice of %d columns does not fit the 16-bit table entries",
              std::max(lds[0], lds[1]));
    return ED_ERR_ARG;
  }
  out.cstart[0] = 0;
  out.cstart[1] = lds[0];
  out.cstart[2] = lds[0] + lds[1];
  out.ld = out.cstart[2];
  DownTables T[2];
  std::vector<int32_t> shop;
  std::vector<uint32_t> sbits;
  for (int sl = 0; sl < 2; ++sl) {
    const int64_t ns = (int64_t)members[sl].size();
    if (ns == 0) {
      T[sl].ld = lds[sl];
      T[sl].rows = 0;
      T[sl].lo.resize((size_t)lds[sl]);
      for (int p = 0; p < lds[sl]; ++p) T[sl].lo[p] = (uint8_t)(p % G);
      continue;
    }
    // the slice's sub-basis: in-slice hops only, targets as local ranks
    shop.assign((size_t)mh * ns, (int32_t)ns);
    sbits.resize((size_t)ns);
    for (int64_t i = 0; i < ns; ++i) {
      const int64_t d = members[sl][i];
      sbits[i] = bits[d];
      int kk = 0;
      for (int k = 0; k < mh; ++k) {
        const uint32_t e = (uint32_t)hop[(size_t)k * n + d];
        const int64_t t = (int64_t)(e & kTargetMask);
        if (t >= n || slice[t] != sl) continue;
        shop[(size_t)kk++ * ns + i] = (int32_t)(((uint32_t)local[t]) | (e & kSignBit));
      }
    }
    const ed_status r = build_down_tables(shop.data(), nullptr, sbits.data(), ns, mh, lds[sl], V, G,
                                          false, T[sl]);
    if (r != ED_OK) return r;
  }
  // columns, bits, slot map
  out.pos.assign((size_t)n, -1);
  out.pad.assign((size_t)out.ld, 0u);
  out.lo.assign((size_t)out.ld, 0);
  std::vector<int64_t> rank_of_col((size_t)out.ld, -1);
  for (int sl = 0; sl < 2; ++sl) {
    for (size_t i = 0; i < members[sl].size(); ++i) {
      const int64_t d = members[sl][i];
      const int col = out.cstart[sl] + T[sl].pos[i];
      out.pos[d] = col;
      out.pad[col] = bits[d];
      rank_of_col[col] = d;
    }
    for (int p = 0; p < lds[sl]; ++p) out.lo[out.cstart[sl] + p] = T[sl].lo[p];
  }
  const int nch = out.ld / CW;
  std::vector<int> xp((size_t)nch, 0), xn((size_t)nch, 0), xpc((size_t)out.ld, 0), xnc((size_t)out.ld, 0);
  for (int p = 0; p < out.ld; ++p) {
    const int64_t d = rank_of_col[p];
    if (d < 0) continue;
    for (int k = 0; k < mh; ++k) {
      const uint32_t e = (uint32_t)hop[(size_t)k * n + d];
      const int64_t t = (int64_t)(e & kTargetMask);
      if (t >= n || slice[t] == slice[d]) continue;
      ++((e & kSignBit) ? xnc : xpc)[p];
    }
    xp[p / CW] = std::max(xp[p / CW], xpc[p]);
    xn[p / CW] = std::max(xn[p / CW], xnc[p]);
  }
  out.rows = std::max(T[0].rows, T[1].rows);
  out.xrows = 0;
  out.kpn.assign(4 * (size_t)nch, 0);
  for (int c = 0; c < nch; ++c) {
    const int sl = c * CW < out.cstart[1] ? 0 : 1;
    const int lc = (c * CW - out.cstart[sl]) / CW;
    if (xp[c] > 255 || xn[c] > 255) {
      set_error("split tables: more than 255 cross-slice hops of one sign");
      return ED_ERR_ARG;
    }
    out.kpn[4 * c] = T[sl].kpn.empty() ? 0 : T[sl].kpn[2 * lc];
    out.kpn[4 * c + 1] = T[sl].kpn.empty() ? 0 : T[sl].kpn[2 * lc + 1];
    out.kpn[4 * c + 2] = (uint8_t)xp[c];
    out.kpn[4 * c + 3] = (uint8_t)xn[c];
    out.xrows = std::max(out.xrows, xp[c] + xn[c]);
  }
  // in-slice entries: the slice's own slots (zero slots ld_s .. ld_s + G - 1)
  out.tab.assign((size_t)std::max(out.rows, 1) * out.ld, 0);
  for (int sl = 0; sl < 2; ++sl)
    for (int k = 0; k < out.rows; ++k)
      for (int p = 0; p < lds[sl]; ++p)
        out.tab[(size_t)k * out.ld + out.cstart[sl] + p] =
            k < T[sl].rows ? T[sl].tab[(size_t)k * lds[sl] + p] : (uint16_t)lds[sl];
  // cross-slice entries: the target's column inside the other slice
  out.xtab.assign((size_t)std::max(out.xrows, 1) * out.ld, 0);
  for (int p = 0; p < out.ld; ++p) {
    const int sl = p < out.cstart[1] ? 0 : 1, o = 1 - sl, c = p / CW;
    const uint16_t zero = (uint16_t)(lds[o] - 1);  // a padding column of the other slice
    for (int k = 0; k < out.xrows; ++k) out.xtab[(size_t)k * out.ld + p] = zero;
    const int64_t d = rank_of_col[p];
    if (d < 0) continue;
    int ip = 0, in = 0;
    for (int k = 0; k < mh; ++k) {
      const uint32_t e = (uint32_t)hop[(size_t)k * n + d];
      const int64_t t = (int64_t)(e & kTargetMask);
      if (t >= n || slice[t] == sl) continue;
      const int row = (e & kSignBit) ? xp[c] + in++ : ip++;
      out.xtab[(size_t)row * out.ld + p] = (uint16_t)(out.pos[t] - out.cstart[o]);
    }
  }
  return ED_OK;
}

}  // namespace ed

extern "C" ed_status ed_hv_split_tables(const int32_t* hop, const uint32_t* bits, int64_t dim,
                                        int32_t maxhops, int32_t V, int32_t G, int32_t site,
                                        uint16_t* table, uint16_t* xtable, int32_t rows_cap,
                                        int32_t cols_cap, int32_t* rows, int32_t* xrows,
                                        int32_t* ld, int32_t* cstart, uint8_t* kpn,
                                        uint8_t* slot_lo, int32_t* colpos) {
  if (!table || !xtable || !rows || !xrows || !ld || !cstart || !kpn || !slot_lo || !colpos) {
    ed::set_error("ed_hv_split_tables: null output");
    return ED_ERR_ARG;
  }
  ed::SplitTables t;
  const ed_status r = ed::build_split_tables(hop, bits, dim, maxhops, V, G, site, t);
  if (r != ED_OK) return r;
  *rows = t.rows;
  *xrows = t.xrows;
  *ld = t.ld;
  if (t.rows > rows_cap || t.xrows > rows_cap || t.ld > cols_cap) {
    ed::set_error("ed_hv_split_tables: %d + %d rows x %d columns, capacity %d x %d", t.rows,
                  t.xrows, t.ld, rows_cap, cols_cap);
    return ED_ERR_ARG;
  }
  std::copy(t.tab.begin(), t.tab.begin() + (size_t)t.rows * t.ld, table);
  std::copy(t.xtab.begin(), t.xtab.begin() + (size_t)t.xrows * t.ld, xtable);
  for (int i = 0; i < 3; ++i) cstart[i] = t.cstart[i];
  std::copy(t.kpn.begin(), t.kpn.end(), kpn);
  std::copy(t.lo.begin(), t.lo.end(), slot_lo);
  std::copy(t.pos.begin(), t.pos.end(), colpos);
  return ED_OK;
}

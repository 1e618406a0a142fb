// Basis construction (Sec. 2.1): combinadic unranking of each species' bit strings and the
// per-state hop tables (target rank + fermion sign), built on the device.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <cmath>
#include <vector>

#include "ed_internal.cuh"

namespace ed {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }

int smem_optin_max() {
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cache[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cache[dev] = v > 0 ? v : 48 * 1024;
  }
  return cache[dev];
}

int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 152;
  if (!cache[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = n > 0 ? n : 152;
  }
  return cache[dev];
}

// ------------------------------------------------------------------ device helpers
// Colex (combinadic) unrank: the state with `n` set bits whose rank among all such
// n_sites-bit integers in ascending order is r. Equivalent to choosing, from the highest
// particle down, the largest position q with C(q, k) <= remaining rank.
__device__ __forceinline__ uint32_t unrank_state(uint64_t r, int n_sites, int n,
                                                 const uint32_t* __restrict__ C) {
  uint32_t s = 0;
  int q = n_sites - 1;
  for (int k = n; k >= 1; --k) {
    while (C[q * kBinomStride + k] > r) --q;  // C(k-1, k) = 0 bounds the loop
    s |= 1u << q;
    r -= C[q * kBinomStride + k];
    --q;
  }
  return s;
}

// Colex rank: sum over the set bits p_1 < p_2 < ... of C(p_k, k).
__device__ __forceinline__ uint32_t rank_state(uint32_t s, const uint32_t* __restrict__ C) {
  uint32_t r = 0;
  int k = 1;
  while (s) {
    int p = __ffs(s) - 1;
    r += C[p * kBinomStride + k];
    ++k;
    s &= s - 1;
  }
  return r;
}

__global__ void unrank_kernel(uint32_t* __restrict__ bits, int64_t dim, int n_sites, int n,
                              const uint32_t* __restrict__ C) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < dim;
       r += (int64_t)gridDim.x * blockDim.x)
    bits[r] = unrank_state((uint64_t)r, n_sites, n, C);
}

// For every state and bond (in bond order) with exactly one occupied end: the hopped
// state, its rank, and the sign (-1)^(occupied sites strictly between the ends).
// With hop == nullptr only counts (max into *maxcount).
__global__ void hop_kernel(const uint32_t* __restrict__ bits, int64_t dim,
                           const int2* __restrict__ bonds, int n_bonds,
                           const uint32_t* __restrict__ C, int32_t* __restrict__ hop,
                           int32_t* __restrict__ hopa, int maxhops, int* __restrict__ maxcount) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < dim;
       r += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t s = bits[r];
    int cnt = 0;
    for (int b = 0; b < n_bonds; ++b) {
      const int i = bonds[b].x, j = bonds[b].y;
      if (((s >> i) ^ (s >> j)) & 1u) {
        if (hop) {
          const int lo = min(i, j), hi = max(i, j);
          const uint32_t between = (uint32_t)((1ull << hi) - 1ull) & ~(uint32_t)((2ull << lo) - 1ull);
          const uint32_t neg = (uint32_t)__popc(s & between) & 1u;
          const uint32_t tgt = rank_state(s ^ ((1u << i) | (1u << j)), C);
          hop[(int64_t)cnt * dim + r] = (int32_t)(tgt | (neg << 31));
          if (hopa) hopa[(int64_t)cnt * dim + r] = 2 * b + (int)((s >> j) & 1u);
        }
        ++cnt;
      }
    }
    if (hop) {
      for (int k = cnt; k < maxhops; ++k) {
        hop[(int64_t)k * dim + r] = (int32_t)dim;
        if (hopa) hopa[(int64_t)k * dim + r] = 0;
      }
    } else {
      atomicMax(maxcount, cnt);
    }
  }
}

constexpr int64_t kMaxOrderedRows = 4000000;  // host RCM up to this many up states

static uint64_t binom_host(int n, int k) {
  if (k < 0 || k > n) return 0;
  uint64_t c = 1;
  for (int i = 1; i <= k; ++i) c = c * (uint64_t)(n - k + i) / (uint64_t)i;
  return c;
}

static ed_status build_species(SpeciesTables& sp, int n_sites, int n, const int2* d_bonds,
                               int n_bonds, const uint32_t* d_binom, int* d_count, bool amps,
                               cudaStream_t s) {
  sp.dim = (int64_t)binom_host(n_sites, n);
  ED_TRY_CUDA(cudaMallocAsync((void**)&sp.bits, sp.dim * sizeof(uint32_t), s));
  const int threads = 256;
  const int64_t want = (sp.dim + threads - 1) / threads;
  const int blocks = (int)(want < 65535 * 8 ? want : 65535 * 8);
  unrank_kernel<<<blocks, threads, 0, s>>>(sp.bits, sp.dim, n_sites, n, d_binom);
  ED_TRY_CUDA(cudaGetLastError());
  ED_TRY_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int), s));
  hop_kernel<<<blocks, threads, 0, s>>>(sp.bits, sp.dim, d_bonds, n_bonds, d_binom, nullptr,
                                        nullptr, 0, d_count);
  ED_TRY_CUDA(cudaGetLastError());
  int h = 0;
  ED_TRY_CUDA(cudaMemcpyAsync(&h, d_count, sizeof(int), cudaMemcpyDeviceToHost, s));
  ED_TRY_CUDA(cudaStreamSynchronize(s));
  sp.maxhops = h;
  if (h > 0) {
    ED_TRY_CUDA(cudaMallocAsync((void**)&sp.hop, (size_t)h * sp.dim * sizeof(int32_t), s));
    if (amps) ED_TRY_CUDA(cudaMallocAsync((void**)&sp.hopa, (size_t)h * sp.dim * sizeof(int32_t), s));
    hop_kernel<<<blocks, threads, 0, s>>>(sp.bits, sp.dim, d_bonds, n_bonds, d_binom, sp.hop,
                                          sp.hopa, h, nullptr);
    ED_TRY_CUDA(cudaGetLastError());
  }
  return ED_OK;
}

// Reverse Cuthill-McKee order of the hop graph of one species (host, from the device
// table): breadth-first search from a low-degree vertex of a far end (two sweeps), each
// vertex's unvisited neighbours taken by increasing degree (ties by index), every
// connected component in turn, the result reversed. Deterministic.
static ed_status rcm_order(const SpeciesTables& sp, cudaStream_t s, std::vector<int32_t>& order) {
  const int64_t n = sp.dim;
  const int mh = sp.maxhops;
  order.resize(n);
  if (mh == 0 || n < 3) {
    for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
    return ED_OK;
  }
  std::vector<int32_t> tab((size_t)mh * n);
  ED_TRY_CUDA(cudaMemcpyAsync(tab.data(), sp.hop, tab.size() * 4, cudaMemcpyDeviceToHost, s));
  ED_TRY_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> deg(n, 0);
  auto nb = [&](int64_t v, int k) { return (int64_t)((uint32_t)tab[(size_t)k * n + v] & kTargetMask); };
  for (int64_t v = 0; v < n; ++v)
    for (int k = 0; k < mh && nb(v, k) < n; ++k) ++deg[v];
  // stamp[v] == cur marks v as visited by the current search; taken[v] marks vertices
  // already placed in the order
  std::vector<int32_t> stamp(n, 0);
  std::vector<char> taken(n, 0);
  int32_t cur = 0;
  std::vector<int32_t> out;
  out.reserve(n);
  std::vector<int32_t> nbuf, visit;
  auto bfs = [&](int64_t root) {
    ++cur;
    visit.clear();
    visit.push_back((int32_t)root);
    stamp[root] = cur;
    for (size_t h = 0; h < visit.size(); ++h) {
      const int64_t v = visit[h];
      nbuf.clear();
      for (int k = 0; k < mh && nb(v, k) < n; ++k) {
        const int64_t w = nb(v, k);
        if (stamp[w] != cur && !taken[w]) {
          stamp[w] = cur;
          nbuf.push_back((int32_t)w);
        }
      }
      std::sort(nbuf.begin(), nbuf.end(), [&](int32_t a, int32_t b) {
        return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
      });
      visit.insert(visit.end(), nbuf.begin(), nbuf.end());
    }
  };
  for (int64_t start = 0; start < n; ++start) {
    if (taken[start]) continue;
    // component of `start`: its lowest-degree vertex, then the last vertex of a search from
    // there (a far end of the component) as the root
    bfs(start);
    int64_t root = visit[0];
    for (int32_t v : visit)
      if (deg[v] < deg[root] || (deg[v] == deg[root] && v < root)) root = v;
    bfs(root);
    bfs(visit.back());
    for (int32_t v : visit) taken[v] = 1;
    out.insert(out.end(), visit.begin(), visit.end());
  }
  for (int64_t i = 0; i < n; ++i) order[i] = out[n - 1 - i];
  return ED_OK;
}

static void free_species(SpeciesTables& sp) {
  if (sp.bits) cudaFree(sp.bits);
  if (sp.hop) cudaFree(sp.hop);
  if (sp.hopa) cudaFree(sp.hopa);
  sp.bits = nullptr;
  sp.hop = nullptr;
  sp.hopa = nullptr;
}

}  // namespace ed

using namespace ed;

extern "C" ed_status ed_build_basis(const ed_lattice* L, int32_t n_up, int32_t n_dn,
                                    void* stream, ed_basis** out) {
  clear_error();
  ED_CHECK_ARG(out != nullptr, "ed_build_basis: out is NULL");
  *out = nullptr;
  ED_CHECK_ARG(L != nullptr, "ed_build_basis: lattice is NULL");
  ED_CHECK_ARG(L->n_sites >= 1 && L->n_sites <= kMaxSites,
               "ed_build_basis: n_sites = %d outside [1, 32]", L->n_sites);
  ED_CHECK_ARG(L->n_bonds >= 0, "ed_build_basis: n_bonds < 0");
  ED_CHECK_ARG(L->n_bonds == 0 || L->bonds != nullptr, "ed_build_basis: bonds is NULL");
  ED_CHECK_ARG(n_up >= 0 && n_up <= L->n_sites && n_dn >= 0 && n_dn <= L->n_sites,
               "ed_build_basis: particle numbers (%d, %d) outside [0, n_sites]", n_up, n_dn);
  std::vector<int2> hb(L->n_bonds > 0 ? L->n_bonds : 1);
  for (int b = 0; b < L->n_bonds; ++b) {
    const int i = L->bonds[2 * b], j = L->bonds[2 * b + 1];
    ED_CHECK_ARG(i >= 0 && i < L->n_sites && j >= 0 && j < L->n_sites && i != j,
                 "ed_build_basis: bond %d = (%d, %d) invalid", b, i, j);
    hb[b] = make_int2(i, j);
  }
  if (L->t_bond)
    for (int b = 0; b < 2 * L->n_bonds; ++b)
      ED_CHECK_ARG(std::isfinite(L->t_bond[b]), "ed_build_basis: t_bond[%d] is not finite", b);
  cudaStream_t s = (cudaStream_t)stream;
  ed_basis* B = new ed_basis();
  cudaGetDevice(&B->device);
  B->n_sites = L->n_sites;
  B->n_up = n_up;
  B->n_dn = n_dn;
  std::vector<uint32_t> C(kBinomStride * kBinomStride);
  for (int n = 0; n <= 32; ++n)
    for (int k = 0; k <= 32; ++k) C[n * kBinomStride + k] = (uint32_t)binom_host(n, k);
  int2* d_bonds = nullptr;
  int* d_count = nullptr;
  ed_status st = ED_OK;
  auto fail = [&](ed_status e) {
    if (d_bonds) cudaFree(d_bonds);
    if (d_count) cudaFree(d_count);
    ed_basis_destroy(B);
    return e;
  };
  if (cudaMalloc((void**)&B->binom, C.size() * sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc((void**)&d_bonds, hb.size() * sizeof(int2)) != cudaSuccess ||
      cudaMalloc((void**)&d_count, sizeof(int)) != cudaSuccess) {
    set_error("ed_build_basis: device allocation failed");
    return fail(ED_ERR_OOM);
  }
  if (cudaMemcpyAsync(B->binom, C.data(), C.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_bonds, hb.data(), hb.size() * sizeof(int2), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    set_error("ed_build_basis: host to device copy failed");
    return fail(ED_ERR_CUDA);
  }
  const bool amps = L->t_bond != nullptr;
  if (amps) {
    B->n_bonds = L->n_bonds;
    if (cudaMalloc((void**)&B->tau, (size_t)(L->n_bonds > 0 ? L->n_bonds : 1) * sizeof(double2)) != cudaSuccess ||
        (L->n_bonds > 0 && cudaMemcpyAsync(B->tau, L->t_bond, (size_t)L->n_bonds * sizeof(double2),
                                           cudaMemcpyHostToDevice, s) != cudaSuccess)) {
      set_error("ed_build_basis: amplitude upload failed");
      return fail(ED_ERR_OOM);
    }
  }
  if ((st = build_species(B->up, L->n_sites, n_up, d_bonds, L->n_bonds, B->binom, d_count, amps, s)) != ED_OK)
    return fail(st);
  if ((st = build_species(B->dn, L->n_sites, n_dn, d_bonds, L->n_bonds, B->binom, d_count, amps, s)) != ED_OK)
    return fail(st);
  B->dim = B->up.dim * B->dn.dim;
  if (B->dn.dim == 1 && B->up.dim > 1) {  // single occupied species: one long row
    std::swap(B->up, B->dn);
    B->swapped = true;
  }
  if (B->up.dim <= kMaxOrderedRows && B->up.maxhops > 0) {
    std::vector<int32_t> order;
    if ((st = rcm_order(B->up, s, order)) != ED_OK) return fail(st);
    if (cudaMalloc((void**)&B->up_order, order.size() * 4) != cudaSuccess ||
        cudaMemcpyAsync(B->up_order, order.data(), order.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      set_error("ed_build_basis: row order upload failed");
      return fail(ED_ERR_CUDA);
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("ed_build_basis: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(ED_ERR_CUDA);
  }
  cudaFree(d_bonds);
  cudaFree(d_count);
  *out = B;
  return ED_OK;
}

extern "C" ed_status ed_basis_dims(const ed_basis* B, int64_t* dim_up, int64_t* dim_dn,
                                   int64_t* dim) {
  clear_error();
  ED_CHECK_ARG(B != nullptr, "ed_basis_dims: basis is NULL");
  if (dim_up) *dim_up = B->user_up().dim;
  if (dim_dn) *dim_dn = B->user_dn().dim;
  if (dim) *dim = B->dim;
  return ED_OK;
}

extern "C" ed_status ed_basis_filling(const ed_basis* B, int32_t* n_sites, int32_t* n_up,
                                      int32_t* n_dn) {
  clear_error();
  ED_CHECK_ARG(B != nullptr, "ed_basis_filling: basis is NULL");
  if (n_sites) *n_sites = B->n_sites;
  if (n_up) *n_up = B->n_up;
  if (n_dn) *n_dn = B->n_dn;
  return ED_OK;
}

extern "C" ed_status ed_basis_tables(const ed_basis* B, const uint32_t** up_bits,
                                     const uint32_t** dn_bits, const int32_t** hop_up,
                                     const int32_t** hop_dn, int32_t* maxhops_up,
                                     int32_t* maxhops_dn) {
  clear_error();
  ED_CHECK_ARG(B != nullptr, "ed_basis_tables: basis is NULL");
  if (up_bits) *up_bits = B->user_up().bits;
  if (dn_bits) *dn_bits = B->user_dn().bits;
  if (hop_up) *hop_up = B->user_up().hop;
  if (hop_dn) *hop_dn = B->user_dn().hop;
  if (maxhops_up) *maxhops_up = B->user_up().maxhops;
  if (maxhops_dn) *maxhops_dn = B->user_dn().maxhops;
  return ED_OK;
}

extern "C" void ed_basis_destroy(ed_basis* B) {
  if (!B) return;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != B->device) cudaSetDevice(B->device);
  lz_cache_free(B);
  hv2_tables_free(B);
  free_species(B->up);
  free_species(B->dn);
  if (B->binom) cudaFree(B->binom);
  if (B->up_order) cudaFree(B->up_order);
  if (B->tau) cudaFree(B->tau);
  if (prev != B->device) cudaSetDevice(prev);
  delete B;
}

extern "C" const char* ed_last_error(void) { return ed::g_err; }

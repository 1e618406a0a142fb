// Host side of the Lanczos-fused H.v (kernel in ed_hv2_kernel.cuh): the variant table, the
// per-plan down tables (column order by hop count and sign, shared-memory slot map), the
// autotuner and the launch.
#include <algorithm>
#include <cstring>
#include <deque>
#include <mutex>
#include <vector>

#include "ed_hv2_kernel.cuh"
#include "ed_hv2c_kernel.cuh"
#include "ed_hv2s_kernel.cuh"
#include "ed_tables.h"

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
  int cst[3] = {0, 0, 0};     // split-row plans: slice starts
  int nslots = 0;             // split-row plans: shared-memory slots (longest slice + G)
  uint16_t* xtab = nullptr;   // split-row plans: cross-slice rows
};

// Split-row variants (hv2s_kernel): id, element, V, T, MB.
#define HV2S_KINDS(X)              \
  X(30, long long, 2, 640, 1)      \
  X(31, float, 4, 512, 2)

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
  if (p->xtab) cudaFree(p->xtab);
  if (p->kpn) cudaFree(p->kpn);
  if (p->slot_lo) cudaFree(p->slot_lo);
  if (p->dn_pad) cudaFree(p->dn_pad);
  if (p->colpos) cudaFree(p->colpos);
  delete p;
}

// Down-state column order and per-geometry tables, built on the host from the basis tables:
// columns ordered by hop count (most first), then by +1-hop count, then by rank; per chunk of
// 32 V columns the table rows [0, kp) hold the +1 hops and [kp, kp + kn) the -1 hops as
// shared-memory slots, each column's hops in the order schedule_gathers gives them.
// Variants with the same (V, G) share them; the basis caches them.
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
  return build_down_tables(hop.data(), hopa.empty() ? nullptr : hopa.data(), bits.data(), n, mh,
                           ld, ki.V, ki.G, cplx, out);
}

static ed_status upload_down_tables(const DownTables& t, int64_t n, cudaStream_t s, Hv2Plan* p) {
  const int ld = t.ld;
  const size_t tbytes = t.cplx ? t.tab32.size() * 4 : t.tab.size() * 2;
  const void* tdata = t.cplx ? (const void*)t.tab32.data() : (const void*)t.tab.data();
  if (cudaMalloc(&p->dtab, tbytes) != cudaSuccess ||
      cudaMalloc((void**)&p->kpn, t.kpn.size()) != cudaSuccess ||
      cudaMalloc((void**)&p->slot_lo, (size_t)ld) != cudaSuccess ||
      cudaMalloc((void**)&p->dn_pad, (size_t)ld * 4) != cudaSuccess ||
      cudaMalloc((void**)&p->colpos, (size_t)(n > 0 ? n : 1) * 4) != cudaSuccess) {
    set_error("H.v tables: out of device memory");
    return ED_ERR_OOM;
  }
  ED_TRY_CUDA(cudaMemcpyAsync(p->dtab, tdata, tbytes, cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaMemcpyAsync(p->kpn, t.kpn.data(), t.kpn.size(), cudaMemcpyHostToDevice, s));
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

void hv2_split_free(const ed_basis* b);
void hv2_tables_free(const ed_basis* b) {
  hv2_split_free(b);
  std::lock_guard<std::mutex> lock(g_tables_mu);
  delete static_cast<std::deque<DownTables>*>(b->hv2_tables);
  b->hv2_tables = nullptr;
}

// ------------------------------------------------------------------ split rows
static std::mutex g_split_mu;
struct SplitCache {
  bool tried = false;
  SplitTables t;
  bool ok = false;
};

static int split_slots(const SplitTables& t) {
  return std::max(t.cstart[1] - t.cstart[0], t.cstart[2] - t.cstart[1]) + t.G;
}

static size_t split_smem(const SplitTables& t, const ed_basis* b, size_t esize) {
  const int MH = b->up.maxhops > 0 ? b->up.maxhops : 1;
  return ((size_t)split_slots(t) * esize + 15) / 16 * 16 + (size_t)MH * 12;
}

// The split tables of this basis for V = 2, G = 16 (int64 kernel) or V = 4, G = 32 (FP32
// kernel), built on first use from the device basis tables and cached on the basis.
static const SplitTables* split_tables(const ed_basis* b, int V, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_split_mu);
  auto* cache = static_cast<SplitCache*>(b->hv2_split);
  if (!cache) b->hv2_split = cache = new SplitCache[2];
  SplitCache& c = cache[V == 2 ? 0 : 1];
  if (!c.tried) {
    c.tried = true;
    const int64_t n = b->dn.dim;
    const int mh = b->dn.maxhops;
    std::vector<int32_t> hop((size_t)mh * n);
    std::vector<uint32_t> bits((size_t)n);
    if ((mh > 0 && cudaMemcpyAsync(hop.data(), b->dn.hop, hop.size() * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
        cudaMemcpyAsync(bits.data(), b->dn.bits, bits.size() * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return nullptr;
    c.ok = build_split_tables(hop.data(), bits.data(), n, mh, V, V == 2 ? 16 : 32, 0, c.t) == ED_OK;
  }
  return c.ok ? &c.t : nullptr;
}

// forced: the caller asked for the split-row variant (schedule 30 / 31) whether or not the
// plain variants fit
static bool split_usable(const ed_basis* b, int mode, int ld_plain, bool forced = false) {
  if (mode != kHv2F32 && mode != kHv2Fx) return false;
  if (b->dn.maxhops > 255 || b->swapped || b->up.dim < 1) return false;
  if (forced) return true;
  if (b->up.dim < kMinRowsStaged) return false;
  // chosen by itself when no plain variant fits, or when the plain ones fit only one CTA per
  // SM (half-rows then run two per SM: 23 ms against 40 ms per H.v on the 18-site FP32 basis)
  static const int pref_f32[] = {1, 4, 2, 6}, pref_fx[] = {8, 9, 12, 11};
  KindInfo ki;
  for (int i = 0; i < 4; ++i)
    if (kind_usable(mode == kHv2Fx ? pref_fx[i] : pref_f32[i], b, mode, ld_plain, &ki) &&
        2 * ki.smem <= (size_t)optin_smem())
      return false;
  return true;
}

int hv2_split_ld(const ed_basis* b, int mode, int schedule, cudaStream_t s) {
  const int ld_plain = (int)((b->dn.dim + 31) / 32 * 32);
  const bool forced = schedule == (mode == kHv2Fx ? 30 : 31);
  if (!split_usable(b, mode, ld_plain, forced)) return 0;
  const SplitTables* t = split_tables(b, mode == kHv2Fx ? 2 : 4, s);
  if (!t) return 0;
  if (split_smem(*t, b, mode == kHv2Fx ? 8 : 4) > (size_t)optin_smem() - 64) return 0;
  return t->ld;
}

void hv2_split_free(const ed_basis* b) {
  std::lock_guard<std::mutex> lock(g_split_mu);
  delete[] static_cast<SplitCache*>(b->hv2_split);
  b->hv2_split = nullptr;
}

static ed_status hv2_build_split(const ed_basis* b, int mode, int ld, cudaStream_t s, Hv2Plan** out) {
  const int V = mode == kHv2Fx ? 2 : 4;
  const SplitTables* t = split_tables(b, V, s);
  if (!t || t->ld != ld) return ED_OK;  // caller falls back to the general kernels
  Hv2Plan* p = new Hv2Plan();
  p->kind = mode == kHv2Fx ? 30 : 31;
  p->smem = split_smem(*t, b, mode == kHv2Fx ? 8 : 4);
  p->ld = ld;
  p->grid = (int)b->up.dim;
  p->nslots = split_slots(*t);
  for (int i = 0; i < 3; ++i) p->cst[i] = t->cstart[i];
  const int64_t n = b->dn.dim;
  if (cudaMalloc(&p->dtab, t->tab.size() * 2) != cudaSuccess ||
      cudaMalloc((void**)&p->xtab, t->xtab.size() * 2) != cudaSuccess ||
      cudaMalloc((void**)&p->kpn, t->kpn.size()) != cudaSuccess ||
      cudaMalloc((void**)&p->slot_lo, (size_t)ld) != cudaSuccess ||
      cudaMalloc((void**)&p->dn_pad, (size_t)ld * 4) != cudaSuccess ||
      cudaMalloc((void**)&p->colpos, (size_t)(n > 0 ? n : 1) * 4) != cudaSuccess) {
    cudaGetLastError();
    hv2_free(p);
    set_error("H.v split tables: out of device memory");
    return ED_ERR_OOM;
  }
  cudaError_t e = cudaMemcpyAsync(p->dtab, t->tab.data(), t->tab.size() * 2, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->xtab, t->xtab.data(), t->xtab.size() * 2, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->kpn, t->kpn.data(), t->kpn.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->slot_lo, t->lo.data(), (size_t)ld, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->dn_pad, t->pad.data(), (size_t)ld * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->colpos, t->pos.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
#define HV2S_ATTR(K, E, V_, T, MB) \
  if (e == cudaSuccess && p->kind == K) e = allow_max_smem(hv2s_kernel<E, V_, T, MB>);
  HV2S_KINDS(HV2S_ATTR)
#undef HV2S_ATTR
  if (e != cudaSuccess) {
    hv2_free(p);
    set_error("H.v split tables: %s", cudaGetErrorString(e));
    return ED_ERR_CUDA;
  }
  *out = p;
  return ED_OK;
}

// Choose the kernel variant for this basis and element type, build the per-plan tables.
ed_status hv2_build(const ed_basis* b, int mode, int ld, int schedule, cudaStream_t s,
                    Hv2Plan** out) {
  *out = nullptr;
  // down-loop lengths are stored in 8 bits
  if (b->dn.maxhops > 255) return ED_OK;  // caller falls back to the general kernels
  if (mode != kHv2C32 &&
      ((schedule == (mode == kHv2Fx ? 30 : 31) &&
        split_usable(b, mode, (int)((b->dn.dim + 31) / 32 * 32), true)) ||
       (schedule < 0 && split_usable(b, mode, (int)((b->dn.dim + 31) / 32 * 32)))))
    return hv2_build_split(b, mode, ld, s, out);
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
  if (!kind) {
    // rows too long for every variant: the split-row kernel, when the stride is its own
    if (split_usable(b, mode, (int)((b->dn.dim + 31) / 32 * 32)))
      return hv2_build_split(b, mode, ld, s, out);
    return ED_OK;  // caller falls back to the general kernels
  }
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
    e = allow_max_smem(hv2_kernel<E, R_, V, T, MB>);
  HV2_KINDS(HV2_ATTR)
#undef HV2_ATTR
#define HV2C_ATTR(K, R_, V, T, MB)                                                         \
  if (kind == K)                                                                          \
    e = allow_max_smem(hv2c_kernel<R_, V, T, MB>);
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
  if (p->kind >= 30) {
    Hv2sArgs c;
    c.up_bits = b->up.bits;
    c.dn_bits = p->dn_pad;
    c.dtab = (const uint16_t*)p->dtab;
    c.xtab = p->xtab;
    c.kpn = reinterpret_cast<const uchar4*>(p->kpn);
    c.slot_lo = p->slot_lo;
    c.hop_up = b->up.hop;
    c.order = b->up_order;
    c.dim_up = b->up.dim;
    c.ld = p->ld;
    c.maxhops_up = b->up.maxhops;
    c.nslots = p->nslots;
    c.cstart0 = p->cst[0];
    c.cstart1 = p->cst[1];
    c.cstart2 = p->cst[2];
    c.t = (float)t;
    c.U = (float)U;
#define HV2S_LAUNCH(K, E, V_, T, MB)                                                          \
    if (p->kind == K)                                                                          \
      hv2s_kernel<E, V_, T, MB><<<p->grid, T, p->smem, s>>>(c, (const E*)x, (E*)y, S, cur, partial);
    HV2S_KINDS(HV2S_LAUNCH)
#undef HV2S_LAUNCH
  }
  if (p->kind >= 20 && p->kind <= 23) {
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

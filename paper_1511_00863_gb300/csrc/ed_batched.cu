// Batched Lanczos (Sec. 2.2, Algorithm 1) over many independent (lattice, filling, U)
// instances in ONE persistent cooperative kernel launch, captured in a CUDA graph.
//
// Instances are packed onto groups of co-resident CTAs by a schedule (kScheds): an instance
// whose dimension reaches a threshold gets a group of several CTAs, smaller instances run
// one after another inside single-CTA groups (only __syncthreads needed there). Groups
// with several CTAs synchronise through a global-memory barrier whose spin is bounded:
// when it runs out the kernel records ED_ERR_TIMEOUT for the batch and returns.
// Per instance and step (FP32 or FP64 vectors, FP64 scalars, as the single-instance ED_F32 /
// ED_F64_NATIVE paths):
//   phase 1: w = s_c H B_c - b_j s_p B_p (written over B_p), partial sums of w . f_j
//   phase 2: a_j, q = w - a_j f_j, partial sums of q . q
//   phase 3: b_{j+1}, scale of f_{j+1}, every `check` steps E0(j) = lambda_min(T_j) by
//            Sturm bisection (leader CTA), convergence / breakdown / max_steps.
// The H.v phase stages blocks of up rows in shared memory (down-hop gathers there) and reads
// up-neighbour rows coalesced; vectors of the batch stay in L2.
// ed_lanczos_solve_batched_mixed carries the FP32 batch to FP64 accuracy: the FP32 run keeps
// its vectors, a Ritz vector is assembled per instance and FP64 steps refine it
// (batched_ritz_kernel and the `refine` form of the FP64 kernel, below).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ed_internal.cuh"
#include "ed_lanczos_dev.cuh"

namespace ed {

constexpr int kBThreads = 256;
// CTAs per SM the register bound allows: the batch is bound by latency across many small
// instances, and 6 CTAs per SM (40 registers, a few words spilled) ran the FP32 batch in 56
// ms against 72 ms with 4 (64 registers). The FP64 kernel keeps 4 (its 64-bit arithmetic
// spills more at 40 registers: 204 ms against 191 ms).
constexpr int kBCtasPerSm = 6;
template <typename T>
constexpr int bctas_per_sm() { return sizeof(T) == 4 ? kBCtasPerSm : 4; }
// Staging area of the H.v phase (a block of up rows, at most kBRowFloats * 4 bytes); the same
// shared buffer holds the leader CTA's bisection workspace at another time.
constexpr int kBRowFloats = 4096;
// Dynamic shared memory of the batched kernels: the row-block staging area, or the bisection
// workspace of T_m for m <= max_steps, whichever is larger (sized per run, so short runs keep
// the L1 data cache that the hop tables are read through).
static size_t bsmem_bytes(int max_steps) {
  const size_t sturm = (size_t)sturm_work_doubles(max_steps + 2) * sizeof(double);
  return sturm > (size_t)kBRowFloats * 4 ? sturm : (size_t)kBRowFloats * 4;
}

struct BInst {
  const uint32_t* upb;
  const uint32_t* dnb;
  const int32_t* hu;
  const int32_t* hd;
  int dim_up, dim_dn, mhu, mhd;
  void* B0;  // two work vectors of the instance (FP32 or FP64 elements)
  void* B1;
  double t, U;
  // mixed solves only: the FP32 phase's Lanczos vectors (raw, [max_steps][dpad]) and the
  // FP64 refinement's two work vectors
  float* V;
  double* D0;
  double* D1;
  int dpad;
};

// Per-instance results and Lanczos scalars (1-based a_j, b_j like LzScalars).
struct BState {
  int j, status;
  double scale[2];
  double tscale;
  double last_E0;
  int last_E0_step;
  int pad_;
};

struct BGroup {
  int first_cta, ncta;
  int inst_begin, inst_end;  // range in the instance order list
};

struct BArgs {
  const BInst* inst;
  BState* st;
  double* alpha;  // [n_inst][max_steps + 2]
  double* beta;   // [n_inst][max_steps + 2]
  double* E0;     // [n_inst][max_steps + 2]
  const int* order;
  const BGroup* groups;
  const int* group_of_cta;
  double* part_a;  // [grid]
  double* part_b;  // [grid]
  unsigned* bar_count;  // [n_groups]
  unsigned* bar_gen;    // [n_groups]
  int* error;
  int max_steps, check;
  double tol;
  uint64_t seed;
  long long max_spin;
  // mixed solves only (batched_ritz_kernel and the refinement): per instance the FP32
  // vectors' scales, y and the inverse iteration's workspace ([n_inst][4 (max_steps + 2)]:
  // vscale | y | 2 (max_steps + 2) of work), the refinement's state and scalars
  BState* st2;
  double* rwork;
  double* alpha2;  // [n_inst][refine_steps + 2]
  double* beta2;
  double* E02;
  int refine_steps;
  double refine_tol;
  int refine;  // batched_lanczos_kernel<double>: run the refinement of a mixed solve
  int store;   // batched_lanczos_kernel<float>: keep the Lanczos vectors (mixed solves)
};

// acc += the signed values of a state's hop targets, hop by hop in table order (so the
// rounding is that of a one-at-a-time loop), taking the table entries and gathered values
// of Q hops before adding any: more loads in flight. tab[k * stride] is hop k's entry; a
// target >= n is padding, and the rest of the state's list is padding too. FP32 takes 4 at
// a time (the 256-instance batch: 51.8 -> 44.3 ms); FP64 one (4 at a time spilled more and
// took 212 against 191 ms).
template <typename T, typename Load>
__device__ __forceinline__ void add_hops(T& acc, const int32_t* tab, int64_t stride, int mh, uint32_t n,
                                         Load load) {
  constexpr int Q = sizeof(T) == 4 ? 4 : 1;
  int k = 0;
  for (; Q > 1 && k + Q <= mh; k += Q) {
    uint32_t en[Q];
    T v[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) en[q] = (uint32_t)tab[(int64_t)(k + q) * stride];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const uint32_t tg = en[q] & kTargetMask;
      v[q] = tg < n ? load(tg) : T(0);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q)
      if ((en[q] & kTargetMask) < n) acc += (en[q] & kSignBit) ? -v[q] : v[q];
    if ((en[Q - 1] & kTargetMask) >= n) return;
  }
  for (; k < mh; ++k) {
    const uint32_t en = (uint32_t)tab[(int64_t)k * stride];
    const uint32_t tg = en & kTargetMask;
    if (tg >= n) return;
    const T v = load(tg);
    acc += (en & kSignBit) ? -v : v;
  }
}

// One instance's run of Algorithm 1, for the CTAs of its group.
struct RunSpec {
  BState* S;
  double* al;
  double* be;
  double* e0;
  void* B0;
  void* B1;
  const double* f1;   // FP64 start vector (unnormalised) or NULL for the seeded one
  float* V;           // store the raw FP32 vector of every step here ([max_steps][dpad]), or NULL
  double* vscale;     // with V: the scale of the stored vector of step j at vscale[j]
  int dpad;
  int max_steps, check;
  double tol;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier of the `g` CTAs of one group. The wait is bounded by `max_spin` nanoseconds of
// the global timer; on expiry (or when another group already failed) it sets *error and
// returns false, and the caller returns from the kernel.
__device__ bool group_barrier(unsigned* count, unsigned* gen, int g, long long max_spin, int* error) {
  __shared__ int ok_s;
  __syncthreads();
  if (g > 1) {
    if (threadIdx.x == 0) {
      int ok = 1;
      const unsigned my_gen = atomicAdd(gen, 0u);
      __threadfence();
      const unsigned arrived = atomicAdd(count, 1u);
      if (arrived == (unsigned)g - 1u) {
        atomicExch(count, 0u);
        __threadfence();
        atomicAdd(gen, 1u);
      } else {
        const unsigned long long t0 = global_ns();
        const long long max_iter = (max_spin >> 6) + 1000000;  // backstop if the timer stalls
        long long it = 0;
        while (atomicAdd(gen, 0u) == my_gen) {
          if ((long long)(global_ns() - t0) > max_spin || ++it > max_iter ||
              *(volatile int*)error != 0) {
            ok = 0;
            atomicExch(error, 1);
            break;
          }
          __nanosleep(128);
        }
      }
      __threadfence();
      ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
  }
  return true;
}

// Loads of data that other CTAs of the group wrote during this launch go to L2 (the L1 of
// this SM is not coherent with their stores).
template <typename T>
__device__ __forceinline__ T ld_shared_f(const T* p, bool multi) { return multi ? __ldcg(p) : *p; }

__device__ __forceinline__ double bstart_element(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
}

// Group-wide sum of the group's CTA partials (fixed order), every thread gets it.
__device__ __forceinline__ double group_sum(const double* part, int first, int g, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < g; i += blockDim.x) v += __ldcg(part + first + i);
  v = block_sum(v, red);
  if (threadIdx.x == 0) red[32] = v;
  __syncthreads();
  v = red[32];
  __syncthreads();
  return v;
}

// T = float (ED_F32) or double (ED_F64_NATIVE): vector elements and H.v arithmetic; the
// scalars are FP64 either way.
// Algorithm 1 for instance I on its group (CTA c of g, leader = c == 0), FP32 or FP64
// vectors T, as specified by R. Returns false when a group barrier's bounded wait ran out.
template <typename T>
__device__ bool run_instance(const BArgs& a, const BInst& I, const RunSpec& R, int c, int g,
                             int first_cta, unsigned* bc, unsigned* bg, double* red, int* stop_s,
                             unsigned char* bsm) {
  constexpr int kRowElems = kBRowFloats * 4 / (int)sizeof(T);  // staged elements of a row block
  T* xsm = reinterpret_cast<T*>(bsm);
  const bool leader = c == 0;
  const bool multi = g > 1;
  BState* S = R.S;
  double* al = R.al;
  double* be = R.be;
  double* e0 = R.e0;
  const int dim = I.dim_up * I.dim_dn;
  const int64_t gt = (int64_t)g * blockDim.x;
  const int64_t t0 = (int64_t)c * blockDim.x + threadIdx.x;
  // ---- start vector: raw values (SplitMix64 or the given FP64 vector), FP64 norm,
  // normalised then rounded
  {
    double v = 0.0;
    for (int64_t e = t0; e < dim; e += gt) {
      const double x = R.f1 ? ld_shared_f(R.f1 + e, multi) : bstart_element(a.seed, (uint64_t)e);
      v = fma(x, x, v);
    }
    v = block_sum(v, red);
    if (threadIdx.x == 0) a.part_a[blockIdx.x] = v;
    if (!group_barrier(bc, bg, g, a.max_spin, a.error)) return false;
    const double inv = 1.0 / sqrt(group_sum(a.part_a, first_cta, g, red));
    for (int64_t e = t0; e < dim; e += gt) {
      const double x = R.f1 ? ld_shared_f(R.f1 + e, multi) : bstart_element(a.seed, (uint64_t)e);
      ((T*)R.B0)[e] = (T)(x * inv);
      ((T*)R.B1)[e] = T(0);
    }
    if (leader && threadIdx.x == 0) {
      S->j = 0;
      S->status = 0;
      S->scale[0] = 1.0;
      S->scale[1] = 0.0;
      S->tscale = 0.0;
      S->last_E0_step = 0;
      S->last_E0 = 0.0;
      be[1] = 0.0;
    }
    if (!group_barrier(bc, bg, g, a.max_spin, a.error)) return false;
  }
  int cur = 0;
  for (int j = 1; j <= R.max_steps; ++j) {
    T* xc = (T*)(cur ? R.B1 : R.B0);
    T* xp = (T*)(cur ? R.B0 : R.B1);
    float* vj = R.V ? R.V + (size_t)(j - 1) * R.dpad : nullptr;
    if (vj && leader && threadIdx.x == 0) R.vscale[j] = __ldcg(&S->scale[cur]);
    // ---- phase 1: fused H.v
    const T sc = (T)__ldcg(&S->scale[cur]);
    const T bsp = (T)(__ldcg(&be[j]) * __ldcg(&S->scale[1 - cur]));
    const T tt = (T)I.t, UU = (T)I.U;
    DotAcc<T> dot;
    if (I.dim_dn <= kRowElems) {
      // blocks of BR consecutive up rows staged in shared memory (coalesced loads; from L2
      // when other CTAs of the group wrote them): down-hop gathers read shared memory,
      // up-hop gathers read whole neighbour rows coalesced
      const int BR = max(1, min(kRowElems, 2048) / I.dim_dn);
      const int nblk = (I.dim_up + BR - 1) / BR;
      for (int blk = c; blk < nblk; blk += g) {
        const int u0 = blk * BR;
        const int nr = min(BR, I.dim_up - u0);
        const int nel = nr * I.dim_dn;
        const T* xb = xc + (int64_t)u0 * I.dim_dn;
        for (int i = threadIdx.x; i < nel; i += blockDim.x) xsm[i] = ld_shared_f(xb + i, multi);
        __syncthreads();
        // (row, column) of element i carried from one iteration to the next: i advances by
        // blockDim.x = sr rows and sd columns
        int r = threadIdx.x / I.dim_dn, d = threadIdx.x - r * I.dim_dn;
        const int sr = blockDim.x / I.dim_dn, sd = blockDim.x - sr * I.dim_dn;
        for (int i = threadIdx.x; i < nel; i += blockDim.x) {
          const int u = u0 + r;
          const T* xr = xsm + r * I.dim_dn;
          T acc = T(0);
          add_hops(acc, I.hd + d, I.dim_dn, I.mhd, (uint32_t)I.dim_dn, [&](uint32_t tg) { return xr[tg]; });
          add_hops(acc, I.hu + u, I.dim_up, I.mhu, (uint32_t)I.dim_up, [&](uint32_t tg) {
            return ld_shared_f(xc + (int64_t)tg * I.dim_dn + d, multi);
          });
          const T xv = xsm[i];
          const int64_t e = (int64_t)u0 * I.dim_dn + i;
          const T hx = fma(-tt, acc, UU * (T)__popc(I.upb[u] & I.dnb[d]) * xv);
          const T w = fma(sc, hx, -bsp * ld_shared_f(xp + e, multi));
          xp[e] = w;
          if (vj) vj[e] = (float)xv;
          dot.add(w, sc * xv);
          r += sr;
          d += sd;
          if (d >= I.dim_dn) {
            d -= I.dim_dn;
            ++r;
          }
        }
        __syncthreads();
      }
    } else {
      // (row, column) of element e carried from one iteration to the next (e < 2^31)
      int u = (int)t0 / I.dim_dn, d = (int)t0 - u * I.dim_dn;
      const int su = (int)gt / I.dim_dn, sdd = (int)gt - su * I.dim_dn;
      for (int64_t e = t0; e < dim; e += gt, u += su, d += sdd) {
        if (d >= I.dim_dn) {
          d -= I.dim_dn;
          ++u;
        }
        const T* xr = xc + (int64_t)u * I.dim_dn;
        T acc = T(0);
        add_hops(acc, I.hd + d, I.dim_dn, I.mhd, (uint32_t)I.dim_dn,
                 [&](uint32_t tg) { return ld_shared_f(xr + tg, multi); });
        add_hops(acc, I.hu + u, I.dim_up, I.mhu, (uint32_t)I.dim_up, [&](uint32_t tg) {
          return ld_shared_f(xc + (int64_t)tg * I.dim_dn + d, multi);
        });
        const T xv = ld_shared_f(xr + d, multi);
        const T hx = fma(-tt, acc, UU * (T)__popc(I.upb[u] & I.dnb[d]) * xv);
        const T w = fma(sc, hx, -bsp * ld_shared_f(xp + e, multi));
        xp[e] = w;
        if (vj) vj[e] = (float)xv;
        dot.add(w, sc * xv);
      }
    }
    {
      const double v = block_sum(dot.get(), red);
      if (threadIdx.x == 0) a.part_a[blockIdx.x] = v;
    }
    if (!group_barrier(bc, bg, g, a.max_spin, a.error)) return false;
    // ---- phase 2: a_j, update
    const double alpha = group_sum(a.part_a, first_cta, g, red);
    if (leader && threadIdx.x == 0) al[j] = alpha;
    const T coef = (T)(alpha * __ldcg(&S->scale[cur]));
    DotAcc<T> q2;
    // (phase 1 wrote w by row blocks: other CTAs' values are read from L2)
    for (int64_t e = t0; e < dim; e += gt) {
      const T q = ld_shared_f(xp + e, multi) - coef * ld_shared_f(xc + e, multi);
      xp[e] = q;
      q2.add(q, q);
    }
    {
      const double v = block_sum(q2.get(), red);
      if (threadIdx.x == 0) a.part_b[blockIdx.x] = v;
    }
    if (!group_barrier(bc, bg, g, a.max_spin, a.error)) return false;
    // ---- phase 3: b_{j+1}, E0(j), stop test (leader), then everyone reads the status
    const double b2 = group_sum(a.part_b, first_cta, g, red);
    if (leader) {
      if (threadIdx.x == 0) {
        const double beta = sqrt(b2);
        const double ts = fmax(S->tscale, fabs(alpha) + be[j]);
        S->tscale = ts;
        be[j + 1] = beta;
        S->j = j;
        int st = (beta > kBreakdownRel * fmax(1.0, ts)) ? 0 : 1;
        if (st == 0) S->scale[1 - cur] = 1.0 / beta;
        *stop_s = st;
      }
      __syncthreads();
      int st = *stop_s;
      if (st != 0 || j >= R.max_steps || (j % R.check) == 0) {
        const double E = sturm_lowest(al, be, j, S->last_E0_step > 0 ? S->last_E0 : NAN,
                                      reinterpret_cast<double*>(bsm), R.max_steps + 2);
        if (threadIdx.x == 0) {
          e0[j] = E;
          if (st == 0 && R.tol > 0.0 && S->last_E0_step > 0 &&
              fabs(E - S->last_E0) <= R.tol * fmax(fabs(E), 1.0))
            st = 2;
          S->last_E0 = E;
          S->last_E0_step = j;
        }
      }
      if (threadIdx.x == 0) {
        if (st == 0 && j >= R.max_steps) st = 3;
        S->status = st;
        __threadfence();
      }
    }
    if (!group_barrier(bc, bg, g, a.max_spin, a.error)) return false;
    if (__ldcg(&S->status) != 0) break;
    cur = 1 - cur;
  }
  return true;
}

template <typename T>
__global__ void __launch_bounds__(kBThreads, bctas_per_sm<T>())
batched_lanczos_kernel(BArgs a) {
  __shared__ double red[33];
  __shared__ int stop_s;
  extern __shared__ __align__(16) unsigned char bsm[];
  const int gi = a.group_of_cta[blockIdx.x];
  const BGroup G = a.groups[gi];
  const int c = blockIdx.x - G.first_cta, g = G.ncta;
  const int stride = a.refine ? a.refine_steps + 2 : a.max_steps + 2;
  for (int oi = G.inst_begin; oi < G.inst_end; ++oi) {
    const int id = a.order[oi];
    const BInst I = a.inst[id];
    RunSpec R;
    if (a.refine) {
      // the FP64 refinement of a mixed solve: from psi, which batched_ritz_kernel left in D1
      R.S = a.st2 + id;
      R.al = a.alpha2 + (size_t)id * stride;
      R.be = a.beta2 + (size_t)id * stride;
      R.e0 = a.E02 + (size_t)id * stride;
      R.B0 = I.D0;
      R.B1 = I.D1;
      R.f1 = I.D1;
      R.max_steps = a.refine_steps;
      R.check = 1;
      R.tol = a.refine_tol;
    } else {
      R.S = a.st + id;
      R.al = a.alpha + (size_t)id * stride;
      R.be = a.beta + (size_t)id * stride;
      R.e0 = a.E0 + (size_t)id * stride;
      R.B0 = I.B0;
      R.B1 = I.B1;
      R.f1 = nullptr;
      R.max_steps = a.max_steps;
      R.check = a.check;
      R.tol = a.tol;
    }
    // mixed solves: the FP32 phase keeps its vectors and their scales (rwork: vscale | y | work)
    R.V = a.store ? I.V : nullptr;
    R.vscale = a.store ? a.rwork + (size_t)id * 4 * stride : nullptr;
    R.dpad = I.dpad;
    if (!run_instance<T>(a, I, R, c, g, G.first_cta, a.bar_count + gi, a.bar_gen + gi, red, &stop_s, bsm))
      return;
  }
}

// Mixed precision per instance (the batched form of ed_lanczos_solve_mixed) in three
// cooperative launches (the first over a plan sized for its kernel's residency, the other two
// over one sized for theirs; all state between them is per instance):
// batched_lanczos_kernel<float> with `store` runs Algorithm 1 in FP32 and keeps its Lanczos
// vectors; batched_ritz_kernel computes the
// eigenvector y of T_m for its lowest eigenvalue (inverse iteration, leader thread) and
// assembles the Ritz vector psi = sum_j y_j f_j into D1; batched_lanczos_kernel<double> with
// `refine` runs Algorithm 1 in FP64 from psi, with E0 checked every step, until the
// refinement's convergence test passes.
__global__ void __launch_bounds__(kBThreads, kBCtasPerSm)
batched_ritz_kernel(BArgs a) {
  __shared__ __align__(16) float coef[ED_MAX_STEPS + 2];  // y_j times the stored vector's scale
  const int gi = a.group_of_cta[blockIdx.x];
  const BGroup G = a.groups[gi];
  const int c = blockIdx.x - G.first_cta, g = G.ncta;
  const bool multi = g > 1;
  const int stride = a.max_steps + 2;
  unsigned* bc = a.bar_count + gi;
  unsigned* bg = a.bar_gen + gi;
  for (int oi = G.inst_begin; oi < G.inst_end; ++oi) {
    const int id = a.order[oi];
    const BInst I = a.inst[id];
    double* rw = a.rwork + (size_t)id * 4 * stride;  // vscale | y | inverse-iteration work (2 strides)
    const double* al = a.alpha + (size_t)id * stride;
    const double* be = a.beta + (size_t)id * stride;
    const int m = __ldcg(&a.st[id].j);
    double* y = rw + stride;
    if (c == 0 && threadIdx.x == 0) {
      if (m >= 1) tridiag_ritz_vector(al, be, m, __ldcg(&a.E0[(size_t)id * stride + m]), y, rw + 2 * stride);
      __threadfence();
    }
    if (!group_barrier(bc, bg, g, a.max_spin, a.error)) return;
    // psi in FP32 arithmetic: it only starts the FP64 refinement, and the FP32 vectors already
    // bound its accuracy far above the FP32 rounding of the sum (GB300's FP64 rate would make
    // this the slowest part of the solve)
    for (int j = 1 + threadIdx.x; j <= m; j += blockDim.x)
      coef[j] = (float)(__ldcg(&y[j]) * __ldcg(&rw[j]));
    __syncthreads();
    const int dim = I.dim_up * I.dim_dn;
    for (int64_t e = (int64_t)c * blockDim.x + threadIdx.x; e < dim; e += (int64_t)g * blockDim.x) {
      float p = 0.f;
      for (int j = 1; j <= m; ++j) p = fmaf(coef[j], ld_shared_f(I.V + (size_t)(j - 1) * I.dpad + e, multi), p);
      I.D1[e] = (double)p;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ schedules
// A schedule maps instances to CTA groups: instances with dim >= big get `gbig` CTAs,
// with dim >= mid get `gmid` CTAs, the rest are queued on single-CTA groups; queues are
// balanced by estimated work (dim x hops x 1), longest first.
// Schedules 5 and 6 instead size groups in proportion to a weight: with T = total weight /
// CTAs, an instance of at least 4096 states and weight w >= 1.5 T gets about w / T CTAs, the
// rest are queued. The weight is the work per step (5), or the work times log2 dim (6), an
// estimate of the steps the instance will take growing with its dimension: a random start
// overlaps the ground state by about dim^-1/2, and the batch's slowest-converging instances
// are its large ones (on the 256-instance batch: FP32 54.8 ms against 56.0 ms with 5; a
// stronger weight, work^1.25, took 71 ms).
struct Sched {
  int big, gbig, mid, gmid;
  int weight;  // proportional schedules: 0 work, 1 work x log2 dim
};
static const Sched kScheds[] = {
    {1 << 30, 1, 1 << 30, 1, 0},  // 0: one CTA per queue, everything queued
    {200000, 8, 20000, 2, 0},     // 1
    {100000, 16, 10000, 4, 0},    // 2
    {400000, 32, 40000, 4, 0},    // 3
    {50000, 8, 5000, 2, 0},       // 4
    {0, 0, 0, 0, 0},              // 5: proportional to work
    {0, 0, 0, 0, 1},              // 6: proportional to work x log2 dim
};
constexpr int kNumScheds = (int)(sizeof(kScheds) / sizeof(kScheds[0]));

struct Plan {
  std::vector<BGroup> groups;
  std::vector<int> group_of_cta;
  std::vector<int> order;
  int grid = 0;
};

static Plan make_plan(const std::vector<long long>& work_in, const std::vector<int>& dims,
                      const Sched& sc, int max_ctas) {
  const int n = (int)dims.size();
  std::vector<long long> work(work_in);
  if (sc.gbig == 0 && sc.weight == 1)
    for (int i = 0; i < n; ++i)
      work[i] = (long long)((double)work_in[i] * std::log2(std::max(2, dims[i])));
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return work[a] != work[b] ? work[a] > work[b] : a < b; });
  Plan p;
  int ctas = 0;
  std::vector<int> big_ids, small_ids;
  const bool prop = sc.gbig == 0;
  std::vector<int> gprop(n, 1);
  if (prop) {
    // T = work per CTA if the batch were spread evenly over all but one CTA; instances of
    // at least 4096 states and 1.5 T get round(w / T) CTAs; the largest groups give CTAs
    // back until the groups fit
    long long W = 0;
    for (long long w : work) W += w;
    const int cap = std::max(1, max_ctas - 1);
    const double T = (double)W / (double)cap;
    long long total = 0;
    for (int i = 0; i < n; ++i) {
      if (dims[i] >= 4096 && (double)work[i] >= 1.5 * T)
        gprop[i] = (int)std::min((double)cap, std::floor((double)work[i] / T + 0.5));
      if (gprop[i] > 1) total += gprop[i];
    }
    while (total > cap) {
      int big = 0;
      for (int i = 1; i < n; ++i)
        if (gprop[i] > gprop[big]) big = i;
      if (gprop[big] <= 1) break;
      --gprop[big];
      --total;
      if (gprop[big] == 1) --total;  // queued from now on
    }
  }
  for (int i : idx) {
    int gsz = dims[i] >= sc.big ? sc.gbig : (dims[i] >= sc.mid ? sc.gmid : 1);
    if (prop) gsz = gprop[i];
    const int cap = prop ? max_ctas - 1 : max_ctas / 2;
    if (gsz > 1 && ctas + gsz <= cap) {
      BGroup G{ctas, gsz, (int)p.order.size(), (int)p.order.size() + 1};
      p.order.push_back(i);
      p.groups.push_back(G);
      ctas += gsz;
    } else {
      small_ids.push_back(i);
    }
  }
  // single-CTA queues for the rest: as many queues as CTAs remain, longest-processing-first
  int nq = std::max(1, std::min((int)small_ids.size(), max_ctas - ctas));
  std::vector<std::vector<int>> q(nq);
  std::vector<long long> load(nq, 0);
  for (int i : small_ids) {
    int best = 0;
    for (int k = 1; k < nq; ++k)
      if (load[k] < load[best]) best = k;
    q[best].push_back(i);
    load[best] += work[i];
  }
  for (int k = 0; k < nq; ++k) {
    if (q[k].empty()) continue;
    BGroup G{ctas, 1, (int)p.order.size(), (int)p.order.size() + (int)q[k].size()};
    for (int i : q[k]) p.order.push_back(i);
    p.groups.push_back(G);
    ctas += 1;
  }
  p.grid = ctas;
  p.group_of_cta.resize(ctas);
  for (int gi = 0; gi < (int)p.groups.size(); ++gi)
    for (int c = 0; c < p.groups[gi].ncta; ++c) p.group_of_cta[p.groups[gi].first_cta + c] = gi;
  return p;
}

// Autotuned schedule per batch signature (dims and hop counts), cached per process.
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune_cache;

}  // namespace ed

using namespace ed;

namespace {

// The FP32 vector store of batched mixed solves (Sum dim x max_steps x 4 bytes, gigabytes for
// a large batch) comes from a per-device memory pool of the library whose release threshold
// keeps the memory reserved after a solve frees it: a repeated solve does not map the store
// again (mapping 12 GB took about 9 ms per call). Process-local; nothing outlasts the process.
cudaMemPool_t vstore_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  uint64_t keep = UINT64_MAX;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  pools[dev] = pool;
  return pool;
}

struct BatchRun {
  int n = 0;
  cudaStream_t stream = nullptr;  // frees the pooled store
  bool pooled = false;
  std::vector<BInst> hinst;
  std::vector<int> dims;
  std::vector<long long> work;
  void* vec = nullptr;
  BInst* d_inst = nullptr;
  BState* d_state = nullptr;
  double* d_scal = nullptr;  // alpha | beta | E0
  int* d_misc = nullptr;     // error flag
  // mixed solves
  bool mixed = false;
  int refine_steps = 0;
  double refine_tol = 0.0;
  void* vstore = nullptr;     // FP32 Lanczos vectors of every instance
  void* dvec = nullptr;       // FP64 refinement vectors
  double* d_rwork = nullptr;
  BState* d_state2 = nullptr;
  double* d_scal2 = nullptr;  // alpha | beta | E0 of the refinement
  ~BatchRun() {
    if (vec) cudaFree(vec);
    if (d_inst) cudaFree(d_inst);
    if (d_state) cudaFree(d_state);
    if (d_scal) cudaFree(d_scal);
    if (d_misc) cudaFree(d_misc);
    if (vstore && pooled) cudaFreeAsync(vstore, stream);
    if (vstore && !pooled) cudaFree(vstore);
    if (dvec) cudaFree(dvec);
    if (d_rwork) cudaFree(d_rwork);
    if (d_state2) cudaFree(d_state2);
    if (d_scal2) cudaFree(d_scal2);
  }
};

struct PlanDev {
  BGroup* groups = nullptr;
  int* goc = nullptr;
  int* order = nullptr;
  double* part = nullptr;
  unsigned* bar = nullptr;
  ~PlanDev() {
    if (groups) cudaFree(groups);
    if (goc) cudaFree(goc);
    if (order) cudaFree(order);
    if (part) cudaFree(part);
    if (bar) cudaFree(bar);
  }
};

ed_status upload_plan(const Plan& p, PlanDev& d, cudaStream_t s) {
  ED_TRY_CUDA(cudaMalloc((void**)&d.groups, p.groups.size() * sizeof(BGroup)));
  ED_TRY_CUDA(cudaMalloc((void**)&d.goc, p.group_of_cta.size() * sizeof(int)));
  ED_TRY_CUDA(cudaMalloc((void**)&d.order, p.order.size() * sizeof(int)));
  ED_TRY_CUDA(cudaMalloc((void**)&d.part, 2 * (size_t)p.grid * sizeof(double)));
  ED_TRY_CUDA(cudaMalloc((void**)&d.bar, 2 * p.groups.size() * sizeof(unsigned)));
  ED_TRY_CUDA(cudaMemcpyAsync(d.groups, p.groups.data(), p.groups.size() * sizeof(BGroup), cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaMemcpyAsync(d.goc, p.group_of_cta.data(), p.group_of_cta.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaMemcpyAsync(d.order, p.order.data(), p.order.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaMemsetAsync(d.bar, 0, 2 * p.groups.size() * sizeof(unsigned), s));
  return ED_OK;
}

// One cooperative launch of the whole batch, captured in a CUDA graph and replayed once.
// p: the plan of the (first) Lanczos launch; p2: the plan of a mixed solve's Ritz and
// refinement launches (their kernels may allow fewer CTAs per SM; all state between the
// launches is per instance, so each launch can pack the instances its own way).
ed_status run_plan(BatchRun& R, const Plan& p, const Plan* p2, const ed_opts* o, int check,
                   cudaStream_t s, float* ms_out) {
  const void* kernel = o->dtype == ED_F64_NATIVE ? (const void*)batched_lanczos_kernel<double>
                                                 : (const void*)batched_lanczos_kernel<float>;
  PlanDev d, d2;
  ed_status st = upload_plan(p, d, s);
  if (st != ED_OK) return st;
  if (R.mixed && (st = upload_plan(*p2, d2, s)) != ED_OK) return st;
  ED_TRY_CUDA(cudaMemsetAsync(R.d_misc, 0, sizeof(int), s));
  BArgs a;
  a.inst = R.d_inst;
  a.st = R.d_state;
  const size_t stride = (size_t)o->max_steps + 2;
  a.alpha = R.d_scal;
  a.beta = R.d_scal + stride * R.n;
  a.E0 = R.d_scal + 2 * stride * R.n;
  a.order = d.order;
  a.groups = d.groups;
  a.group_of_cta = d.goc;
  a.part_a = d.part;
  a.part_b = d.part + p.grid;
  a.bar_count = d.bar;
  a.bar_gen = d.bar + p.groups.size();
  a.error = R.d_misc;
  a.max_steps = o->max_steps;
  a.check = check;
  a.tol = o->tol;
  a.seed = o->seed;
  a.max_spin = 1000000000LL;  // a group barrier waits at most 1 s
  a.st2 = R.d_state2;
  a.rwork = R.d_rwork;
  const size_t stride2 = (size_t)R.refine_steps + 2;
  a.alpha2 = R.d_scal2;
  a.beta2 = R.d_scal2 ? R.d_scal2 + stride2 * R.n : nullptr;
  a.E02 = R.d_scal2 ? R.d_scal2 + 2 * stride2 * R.n : nullptr;
  a.refine_steps = R.refine_steps;
  a.refine_tol = R.refine_tol;
  a.refine = 0;
  a.store = R.mixed ? 1 : 0;
  BArgs ar = a;  // mixed solves: the Ritz launch and the FP64 refinement over plan p2
  if (R.mixed) {
    ar.order = d2.order;
    ar.groups = d2.groups;
    ar.group_of_cta = d2.goc;
    ar.part_a = d2.part;
    ar.part_b = d2.part + p2->grid;
    ar.bar_count = d2.bar;
    ar.bar_gen = d2.bar + p2->groups.size();
  }
  ar.store = 0;
  BArgs a2 = ar;
  a2.refine = 1;
  void* args[] = {&a};
  void* argsr[] = {&ar};
  void* args2[] = {&a2};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ED_TRY_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  const size_t dsm = bsmem_bytes(o->max_steps), dsm2 = bsmem_bytes(R.refine_steps);
  cudaError_t le = cudaLaunchCooperativeKernel(kernel, p.grid, kBThreads, args, dsm, s);
  if (le == cudaSuccess && R.mixed)
    le = cudaLaunchCooperativeKernel((const void*)batched_ritz_kernel, p2->grid, kBThreads, argsr, 0, s);
  if (le == cudaSuccess && R.mixed)
    le = cudaLaunchCooperativeKernel((const void*)batched_lanczos_kernel<double>, p2->grid, kBThreads,
                                     args2, dsm2, s);
  cudaError_t ce = cudaStreamEndCapture(s, &graph);
  if (le != cudaSuccess || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    set_error("batched Lanczos: capture of the cooperative launch failed: %s",
              cudaGetErrorString(le != cudaSuccess ? le : ce));
    return ED_ERR_CUDA;
  }
  cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    set_error("batched Lanczos: graph instantiate failed: %s", cudaGetErrorString(ie));
    return ED_ERR_CUDA;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  cudaError_t ge = cudaGraphLaunch(exec, s);
  cudaEventRecord(e1, s);
  cudaError_t se = cudaStreamSynchronize(s);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(exec);
  if (ge != cudaSuccess || se != cudaSuccess) {
    set_error("batched Lanczos: %s", cudaGetErrorString(ge != cudaSuccess ? ge : se));
    return ED_ERR_CUDA;
  }
  int err = 0;
  ED_TRY_CUDA(cudaMemcpy(&err, R.d_misc, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    set_error("batched Lanczos: a group barrier timed out");
    return ED_ERR_TIMEOUT;
  }
  if (ms_out) *ms_out = ms;
  return ED_OK;
}

}  // namespace

namespace ed {
// Self-test kernel of the bounded group barrier: CTA `absent` never arrives, so the other
// CTAs of the group must give up after `limit_ns` and flag the error.
__global__ void barrier_selftest_kernel(unsigned* bar, int* error, int absent, long long limit_ns) {
  if ((int)blockIdx.x == absent) return;
  group_barrier(bar, bar + 1, gridDim.x, limit_ns, error);
}
}  // namespace ed

extern "C" ed_status ed_selftest_barrier_timeout(int32_t ctas, int32_t timeout_ms, void* stream) {
  clear_error();
  ED_CHECK_ARG(ctas >= 2 && ctas <= 64 && timeout_ms >= 1 && timeout_ms <= 5000,
               "ed_selftest_barrier_timeout: ctas in [2, 64], timeout_ms in [1, 5000]");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* bar = nullptr;
  int* err = nullptr;
  struct ReleaseOnReturn {  // frees the scratch on every return path, error returns included
    cudaStream_t s;
    unsigned*& bar;
    int*& err;
    ~ReleaseOnReturn() {
      if (bar) cudaFreeAsync(bar, s);
      if (err) cudaFreeAsync(err, s);
    }
  } release{s, bar, err};
  ED_TRY_CUDA(cudaMallocAsync((void**)&bar, 2 * sizeof(unsigned), s));
  ED_TRY_CUDA(cudaMallocAsync((void**)&err, sizeof(int), s));
  ED_TRY_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
  ED_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  int absent = ctas - 1;
  long long limit = (long long)timeout_ms * 1000000LL;
  void* args[] = {&bar, &err, &absent, &limit};
  ED_TRY_CUDA(cudaLaunchCooperativeKernel((const void*)barrier_selftest_kernel, ctas, 32, args, 0, s));
  int h = 0;
  ED_TRY_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  ED_TRY_CUDA(cudaStreamSynchronize(s));
  if (h) {
    set_error("group barrier wait ran out after %d ms (as the self-test intends)", timeout_ms);
    return ED_ERR_TIMEOUT;
  }
  return ED_OK;
}

static ed_status solve_batched(int32_t n, const ed_basis* const* bases, const ed_params* params,
                               const ed_opts* o, bool mixed, int32_t refine_steps, double refine_tol,
                               void* stream, double* E0, int32_t* steps, int32_t* steps64,
                               int32_t* status, int32_t* schedule_used) {
  const char* fn = mixed ? "ed_lanczos_solve_batched_mixed" : "ed_lanczos_solve_batched";
  ED_CHECK_ARG(n >= 1 && bases && params && o && E0, "%s: bad arguments", fn);
  if (mixed)
    ED_CHECK_ARG(o->dtype == ED_F32, "%s: dtype must be ED_F32 (the phase before refinement)", fn);
  else
    ED_CHECK_ARG(o->dtype == ED_F32 || o->dtype == ED_F64_NATIVE,
                 "%s: dtype must be ED_F32 or ED_F64_NATIVE", fn);
  ED_CHECK_ARG(o->reorth == 0, "%s: reorth must be 0 (none)", fn);
  ED_CHECK_ARG(o->max_steps >= 1 && o->max_steps <= ED_MAX_STEPS, "max_steps out of range");
  ED_CHECK_ARG(!mixed || (refine_steps >= 1 && refine_steps <= ED_MAX_STEPS),
               "%s: refine_steps out of range", fn);
  ED_CHECK_ARG(o->schedule >= -1 && o->schedule < kNumScheds, "schedule %d out of range", o->schedule);
  cudaStream_t user = (cudaStream_t)stream;
  cudaStream_t s = nullptr;
  ED_TRY_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamDestroy(s); }
  } guard{s};
  {
    cudaEvent_t ev;
    ED_TRY_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEventRecord(ev, user);
    cudaStreamWaitEvent(s, ev, 0);
    cudaEventDestroy(ev);
  }
  BatchRun R;
  R.n = n;
  R.hinst.resize(n);
  R.dims.resize(n);
  R.work.resize(n);
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    const ed_basis* b = bases[i];
    ED_CHECK_ARG(b != nullptr, "%s: basis %d is NULL", fn, i);
    ED_CHECK_ARG(!b->has_tau(), "%s: basis %d has complex amplitudes", fn, i);
    ED_CHECK_ARG(b->dim < (1LL << 31), "%s: instance %d too large", fn, i);
    R.dims[i] = (int)b->dim;
    R.work[i] = (long long)b->dim * (b->up.maxhops + b->dn.maxhops + 4);
    total += (size_t)((b->dim + 3) / 4 * 4);
  }
  const size_t esize = o->dtype == ED_F64_NATIVE ? 8 : 4;
  const size_t stride = (size_t)o->max_steps + 2;
  ED_TRY_CUDA(cudaMalloc((void**)&R.vec, 2 * total * esize));
  if (mixed) {
    R.mixed = true;
    R.refine_steps = refine_steps;
    R.refine_tol = refine_tol;
    const size_t stride2 = (size_t)refine_steps + 2;
    const size_t vbytes = total * (size_t)o->max_steps * sizeof(float);
    cudaMemPool_t pool = vstore_pool();
    R.stream = s;
    const cudaError_t ve = pool ? cudaMallocFromPoolAsync(&R.vstore, vbytes, pool, s)
                                : cudaMalloc(&R.vstore, vbytes);
    if (ve != cudaSuccess) {
      cudaGetLastError();
      R.vstore = nullptr;
      set_error("%s: %zu bytes for the FP32 Lanczos vectors are not available", fn, vbytes);
      return ED_ERR_OOM;
    }
    R.pooled = pool != nullptr;
    ED_TRY_CUDA(cudaMalloc(&R.dvec, 2 * total * sizeof(double)));
    ED_TRY_CUDA(cudaMalloc((void**)&R.d_rwork, 4 * stride * n * sizeof(double)));
    ED_TRY_CUDA(cudaMalloc((void**)&R.d_state2, n * sizeof(BState)));
    ED_TRY_CUDA(cudaMalloc((void**)&R.d_scal2, 3 * stride2 * n * sizeof(double)));
    ED_TRY_CUDA(cudaMemsetAsync(R.d_scal2, 0, 3 * stride2 * n * sizeof(double), s));
    ED_TRY_CUDA(cudaMemsetAsync(R.d_rwork, 0, 4 * stride * n * sizeof(double), s));
  }
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    const ed_basis* b = bases[i];
    BInst& I = R.hinst[i];
    I.upb = b->up.bits;
    I.dnb = b->dn.bits;
    I.hu = b->up.hop;
    I.hd = b->dn.hop;
    I.dim_up = (int)b->up.dim;
    I.dim_dn = (int)b->dn.dim;
    I.mhu = b->up.maxhops;
    I.mhd = b->dn.maxhops;
    const size_t dpad = (size_t)(b->dim + 3) / 4 * 4;
    I.dpad = (int)dpad;
    // the two work vectors of an instance side by side (per instance: B0, B1; D0, D1)
    I.B0 = (char*)R.vec + 2 * off * esize;
    I.B1 = (char*)R.vec + (2 * off + dpad) * esize;
    I.V = mixed ? (float*)R.vstore + off * (size_t)o->max_steps : nullptr;
    I.D0 = mixed ? (double*)R.dvec + 2 * off : nullptr;
    I.D1 = mixed ? (double*)R.dvec + 2 * off + dpad : nullptr;
    off += dpad;
    I.t = params[i].t;
    I.U = params[i].U;
  }
  ED_TRY_CUDA(cudaMalloc((void**)&R.d_inst, n * sizeof(BInst)));
  ED_TRY_CUDA(cudaMalloc((void**)&R.d_state, n * sizeof(BState)));
  ED_TRY_CUDA(cudaMalloc((void**)&R.d_scal, 3 * stride * n * sizeof(double)));
  ED_TRY_CUDA(cudaMalloc((void**)&R.d_misc, sizeof(int)));
  ED_TRY_CUDA(cudaMemcpyAsync(R.d_inst, R.hinst.data(), n * sizeof(BInst), cudaMemcpyHostToDevice, s));
  ED_TRY_CUDA(cudaMemsetAsync(R.d_scal, 0, 3 * stride * n * sizeof(double), s));

  // a cooperative launch needs every CTA resident: grids of (resident CTAs per SM) x SMs
  int per_sm = 0, per_sm2 = 0;
  if (o->dtype == ED_F64_NATIVE)
    ED_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_lanczos_kernel<double>,
                                                              kBThreads, bsmem_bytes(o->max_steps)));
  else
    ED_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_lanczos_kernel<float>,
                                                              kBThreads, bsmem_bytes(o->max_steps)));
  if (mixed) {  // the Ritz and refinement launches share a plan
    int pm = 0, pd = 0;
    ED_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pm, batched_ritz_kernel, kBThreads, 0));
    ED_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pd, batched_lanczos_kernel<double>,
                                                              kBThreads, bsmem_bytes(refine_steps)));
    per_sm2 = std::min(pm, pd);
  }
  ED_CHECK_ARG(per_sm >= 1 && (!mixed || per_sm2 >= 1), "%s: the batched kernels do not fit an SM", fn);
  const int max_ctas = sm_count() * std::min(per_sm, o->dtype == ED_F64_NATIVE
                                                         ? bctas_per_sm<double>() : bctas_per_sm<float>());
  const int max_ctas2 = sm_count() * std::min(std::max(per_sm2, 1), kBCtasPerSm);
  const int check = 4;  // E0(j) every 4 steps (and at the stop step)
  int sched = o->schedule;
  if (sched < 0) {
    // autotune: time every candidate schedule on this batch with a short plain run (the
    // schedules pack the same H.v work in both forms), keep the best
    std::string key;
    for (int i = 0; i < n; ++i) key += std::to_string(R.work[i]) + ",";
    key += std::to_string(max_ctas) + "/" + std::to_string((int)o->dtype);
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) sched = it->second;
    }
    if (sched < 0) {
      // the real solve (its tolerance, at most 200 steps): how instances converge decides
      // the batch's tail as much as the work per step does
      ed_opts ot = *o;
      ot.max_steps = std::min(o->max_steps, 200);
      const bool was_mixed = R.mixed;
      R.mixed = false;
      float best = 1e30f;
      for (int k = 0; k < kNumScheds; ++k) {
        const Plan p = make_plan(R.work, R.dims, kScheds[k], max_ctas);
        float ms = 0.f;
        ed_status r = run_plan(R, p, nullptr, &ot, check, s, &ms);
        if (r != ED_OK) return r;
        if (ms < best) best = ms, sched = k;
      }
      R.mixed = was_mixed;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = sched;
    }
  }
  const Plan p = make_plan(R.work, R.dims, kScheds[sched], max_ctas);
  const Plan p2 = mixed ? make_plan(R.work, R.dims, kScheds[sched], max_ctas2) : Plan();
  float ms = 0.f;
  ed_status r = run_plan(R, p, mixed ? &p2 : nullptr, o, check, s, &ms);
  if (r != ED_OK) return r;
  std::vector<BState> hs(n), hs2(mixed ? n : 0);
  ED_TRY_CUDA(cudaMemcpy(hs.data(), R.d_state, n * sizeof(BState), cudaMemcpyDeviceToHost));
  const size_t stride_out = mixed ? (size_t)refine_steps + 2 : stride;
  std::vector<double> hE(stride_out * n);
  if (mixed) {
    ED_TRY_CUDA(cudaMemcpy(hs2.data(), R.d_state2, n * sizeof(BState), cudaMemcpyDeviceToHost));
    ED_TRY_CUDA(cudaMemcpy(hE.data(), R.d_scal2 + 2 * stride_out * n, stride_out * n * sizeof(double),
                           cudaMemcpyDeviceToHost));
  } else {
    ED_TRY_CUDA(cudaMemcpy(hE.data(), R.d_scal + 2 * stride * n, stride * n * sizeof(double),
                           cudaMemcpyDeviceToHost));
  }
  bool all_conv = true;
  for (int i = 0; i < n; ++i) {
    const BState& F = mixed ? hs2[i] : hs[i];
    const int j = F.j;
    E0[i] = j >= 1 ? hE[(size_t)i * stride_out + j] : NAN;
    if (steps) steps[i] = hs[i].j;
    if (steps64) steps64[i] = mixed ? hs2[i].j : 0;
    if (status) status[i] = F.status;
    if (F.status == 3 && (mixed ? refine_tol : o->tol) > 0.0) all_conv = false;
  }
  if (schedule_used) *schedule_used = sched;
  if (!all_conv) {
    set_error("%s: some instances reached max_steps before converging", fn);
    return ED_ERR_NOT_CONVERGED;
  }
  return ED_OK;
}

extern "C" ed_status ed_lanczos_solve_batched(int32_t n, const ed_basis* const* bases,
                                              const ed_params* params, const ed_opts* o,
                                              void* stream, double* E0, int32_t* steps,
                                              int32_t* status, int32_t* schedule_used) {
  clear_error();
  return solve_batched(n, bases, params, o, false, 0, 0.0, stream, E0, steps, nullptr, status,
                       schedule_used);
}

extern "C" ed_status ed_lanczos_solve_batched_mixed(int32_t n, const ed_basis* const* bases,
                                                    const ed_params* params, const ed_opts* o,
                                                    int32_t refine_steps, double refine_tol,
                                                    void* stream, double* E0, int32_t* steps32,
                                                    int32_t* steps64, int32_t* status,
                                                    int32_t* schedule_used) {
  clear_error();
  return solve_batched(n, bases, params, o, true, refine_steps, refine_tol, stream, E0, steps32,
                       steps64, status, schedule_used);
}

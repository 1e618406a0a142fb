// Learned Lanczos start vector: a small network over the occupation bits of a basis state
// (and U) predicts the ground-state amplitude; its predictions over the whole basis become
// f_1 of Algorithm 1 (Sec. 2.2). The paper has no learned component.
//
//   x = (up bits, down bits, bf16(U/8)) in R^(2L+1); h1 = tanh(W1^T x + b1);
//   h2 = tanh(W2^T bf16(h1) + b2);
//   (a, z) = W3^T h2 + b3; psi0 = sign(z) exp(a).       64 hidden units per layer.
// Weights: FP32 master copy (Adam, Kingma & Ba 2015), rounded to bfloat16 (nearest even)
// for every forward pass; FP32 accumulation. The U feature and the first layer's output
// enter the next product rounded to bfloat16 (the operands of the tensor-core products of
// the inference kernel); the backward pass treats these roundings as the identity.
// Inference evaluates tanh with the special-function unit's approximation (PTX
// tanh.approx.f32, maximum relative error about 2^-11: one instruction instead of the ~19 of
// an accurate tanhf, which made the inference issue-bound); training uses tanhf. The
// predicted vector only starts Algorithm 1, so an error of that size in the activations
// changes nothing the method relies on.
// Training: samples drawn uniformly from the basis with weight dim * psi^2; loss per sample
// (a - log|psi|)^2 + log(1 + exp(-sign(psi) z)); deterministic per-CTA gradient partials
// reduced in a fixed order.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ed_internal.cuh"
#include "ed_tcgen05.cuh"

namespace ed {

constexpr int kH = 64;         // hidden units
constexpr int kMaxIn = 2 * kMaxSites + 1;
constexpr int kTile = 64;      // samples per tile in the training kernel
constexpr int kMThreads = 256;

struct MlpDims {
  int L, nin;
  int oW1, ob1, oW2, ob2, oW3, ob3, P;
};

__host__ __device__ inline MlpDims mlp_dims(int L) {
  MlpDims d;
  d.L = L;
  d.nin = 2 * L + 1;
  d.oW1 = 0;
  d.ob1 = d.oW1 + d.nin * kH;
  d.oW2 = d.ob1 + kH;
  d.ob2 = d.oW2 + kH * kH;
  d.oW3 = d.ob2 + kH;
  d.ob3 = d.oW3 + kH * 2;
  d.P = d.ob3 + 2;
  return d;
}

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// tanh on the special-function unit (PTX tanh.approx.f32, sm_75 and later)
__device__ __forceinline__ float tanh_sfu(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Rounded weights into shared memory (sw has P floats).
__device__ __forceinline__ void load_weights(const float* __restrict__ params, int P, float* sw) {
  for (int i = threadIdx.x; i < P; i += blockDim.x) sw[i] = bf16r(params[i]);
  __syncthreads();
}

// ------------------------------------------------------------------ inference
// 5th-generation tensor cores: a CTA of 4 warps evaluates tiles of 128 basis states, one
// state per thread (TMEM lane). The features of the tile (bits as 0/1, bf16(U/8), zero
// padding to K1 = 16 ceil(nin/16)) and later bf16(h1) are written to shared memory in the
// K-major core-matrix layout; one thread issues tcgen05.mma (BF16 x BF16 -> FP32 in TMEM
// columns 0..63: D1 = X W1, then D2 = bf16(h1) W2 over it, once every thread has read D1)
// and commits to an mbarrier; every thread then reads its row of the accumulator with
// tcgen05.ld and applies
// bias (CUDA cores) and tanh (special-function unit); the 64 -> 2 output layer stays on the
// CUDA cores.
// Waits on the mbarrier are bounded (1 s of the global timer); on expiry the kernel sets
// *err, frees its TMEM and returns.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

constexpr int kTcRows = 128;      // states per tile = threads per CTA = TMEM lanes used
constexpr uint32_t kTcCols = 64;   // TMEM columns of D1, then of D2
// At most 8 CTAs per SM (8 x 64 = all 512 TMEM columns, so no allocation ever waits): with
// 1 KB reserved per CTA, 9 x (25 KB + 1 KB) exceeds the SM's 228 KB. The register bound
// (launch bounds) makes 5 resident; the grid is one wave of them.
constexpr int kTcSmemMin = 25600;
constexpr int kTcCtasPerSm = 5;

struct TcLayout {
  int K1;
  uint32_t a1, a2, b1, b2, par, mbar, tslot, total;
};

__host__ __device__ inline TcLayout tc_layout(int nin) {
  auto up = [](uint32_t v, uint32_t a) { return (v + a - 1) / a * a; };
  TcLayout t;
  t.K1 = (nin + 15) / 16 * 16;
  t.a1 = 0;
  t.a2 = up(t.a1 + (uint32_t)kTcRows * t.K1 * 2, 1024);
  t.b1 = up(t.a2 + (uint32_t)kTcRows * kH * 2, 1024);
  t.b2 = up(t.b1 + (uint32_t)kH * t.K1 * 2, 1024);
  t.par = up(t.b2 + (uint32_t)kH * kH * 2, 1024);
  t.mbar = up(t.par + (uint32_t)(4 * kH + 2) * 4, 16);
  t.tslot = t.mbar + 8;
  t.total = up(t.tslot + 8, 1024);
  return t;
}

template <typename T>
__global__ void __launch_bounds__(kTcRows, kTcCtasPerSm)
mlp_infer_tc_kernel(const float* __restrict__ params, int L, float U, const uint32_t* __restrict__ upb,
                    const uint32_t* __restrict__ dnb, int64_t dim_dn, int64_t dim, T* __restrict__ out,
                    int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  const MlpDims d = mlp_dims(L);
  const TcLayout ly = tc_layout(d.nin);
  const int K1 = ly.K1;
  unsigned char* A1 = tsm + ly.a1;
  unsigned char* A2 = tsm + ly.a2;
  unsigned char* B1 = tsm + ly.b1;
  unsigned char* B2 = tsm + ly.b2;
  float* sb1 = reinterpret_cast<float*>(tsm + ly.par);
  float* sb2 = sb1 + kH;
  float* sW3 = sb2 + kH;
  float* sb3 = sW3 + 2 * kH;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tsm + ly.tslot);
  const uint32_t mbar = smem_addr(tsm + ly.mbar);
  const int tid = threadIdx.x, warp = tid >> 5;

  // rounded weights: W1, W2 as K-major B operands (row n = output unit), the rest in FP32
  for (int i = tid; i < kH * K1; i += blockDim.x) {
    const int n = i / K1, k = i - n * K1;
    const float w = k < d.nin ? params[d.oW1 + k * kH + n] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(B1 + cm_offset(n, k, K1)) = __float2bfloat16_rn(w);
  }
  for (int i = tid; i < kH * kH; i += blockDim.x) {
    const int n = i / kH, k = i - n * kH;
    *reinterpret_cast<__nv_bfloat16*>(B2 + cm_offset(n, k, kH)) =
        __float2bfloat16_rn(params[d.oW2 + k * kH + n]);
  }
  for (int i = tid; i < kH; i += blockDim.x) {
    sb1[i] = bf16r(params[d.ob1 + i]);
    sb2[i] = bf16r(params[d.ob2 + i]);
    sW3[2 * i] = bf16r(params[d.oW3 + 2 * i]);
    sW3[2 * i + 1] = bf16r(params[d.oW3 + 2 * i + 1]);
  }
  if (tid < 2) sb3[tid] = bf16r(params[d.ob3 + tid]);
  if (tid == 0) mbar_init(mbar, 1);
  if (warp == 0) tc_alloc(smem_addr(tslot), kTcCols);
  fence_smem_to_async();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t lanes = (uint32_t)(warp * 32) << 16;  // this warp's TMEM lane quarter
  const float u8 = bf16r(U * 0.125f);
  const uint32_t idesc = tc_idesc_bf16_f32(kTcRows, kH);
  const uint32_t a1s = smem_addr(A1), a2s = smem_addr(A2), b1s = smem_addr(B1), b2s = smem_addr(B2);
  const uint32_t sbo1 = (uint32_t)(K1 >> 3) << 7, sbo2 = (uint32_t)(kH >> 3) << 7;
  constexpr unsigned long long kWaitNs = 1000000000ull;
  uint32_t phase = 0;
  bool ok = true;
  const int64_t ntiles = (dim + kTcRows - 1) / kTcRows;
  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int64_t e = tile * kTcRows + tid;
    const bool valid = e < dim;
    uint32_t ub = 0, db = 0;
    if (valid) {
      const int64_t u = e / dim_dn;
      ub = upb[u];
      db = dnb[e - u * dim_dn];
    }
    auto feat = [&](int f) -> float {
      if (f < L) return (float)((ub >> f) & 1u);
      if (f < 2 * L) return (float)((db >> (f - L)) & 1u);
      return f == 2 * L ? u8 : 0.f;
    };
    for (int j = 0; j < K1; j += 8) {
      const uint4 w = make_uint4(pack_bf16(feat(j), feat(j + 1)), pack_bf16(feat(j + 2), feat(j + 3)),
                                 pack_bf16(feat(j + 4), feat(j + 5)), pack_bf16(feat(j + 6), feat(j + 7)));
      *reinterpret_cast<uint4*>(A1 + cm_offset(tid, j, K1)) = w;
    }
    // ---- layer 1 on the tensor cores
    fence_smem_to_async();
    tc_fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after_sync();
      for (int s = 0; s < K1 / 16; ++s)
        tc_mma_f16(tmem, tc_smem_desc(a1s + s * 256, 128, sbo1), tc_smem_desc(b1s + s * 256, 128, sbo1),
                   idesc, s > 0);
      tc_commit(mbar);
    }
    ok = __syncthreads_and(mbar_wait_bounded(mbar, phase, kWaitNs)) != 0;
    phase ^= 1u;
    if (!ok) break;
    tc_fence_after_sync();
    float h[kH];
    tc_ld32(tmem + lanes, h);
    tc_ld32(tmem + lanes + 32, h + 32);
#pragma unroll
    for (int j = 0; j < kH; j += 8) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        w[q] = pack_bf16(tanh_sfu(h[j + 2 * q] + sb1[j + 2 * q]),
                         tanh_sfu(h[j + 2 * q + 1] + sb1[j + 2 * q + 1]));
      *reinterpret_cast<uint4*>(A2 + cm_offset(tid, j, kH)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    // ---- layer 2 on the tensor cores
    fence_smem_to_async();
    tc_fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after_sync();
      for (int s = 0; s < kH / 16; ++s)
        tc_mma_f16(tmem, tc_smem_desc(a2s + s * 256, 128, sbo2), tc_smem_desc(b2s + s * 256, 128, sbo2),
                   idesc, s > 0);
      tc_commit(mbar);
    }
    ok = __syncthreads_and(mbar_wait_bounded(mbar, phase, kWaitNs)) != 0;
    phase ^= 1u;
    if (!ok) break;
    tc_fence_after_sync();
    tc_ld32(tmem + lanes, h);
    tc_ld32(tmem + lanes + 32, h + 32);
    // ---- output layer on the CUDA cores
    float a = sb3[0], z = sb3[1];
#pragma unroll
    for (int n = 0; n < kH; ++n) {
      const float t = tanh_sfu(h[n] + sb2[n]);
      a = fmaf(t, sW3[2 * n], a);
      z = fmaf(t, sW3[2 * n + 1], z);
    }
    if (valid) {
      const float v = expf(a);
      out[e] = (T)(z >= 0.f ? v : -v);
    }
    tc_fence_before_sync();  // this tile's TMEM reads before the next tile's MMAs
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after_sync();
    tc_dealloc(tmem, kTcCols);
  }
}

// ------------------------------------------------------------------ loss and gradient
// Each CTA walks tiles of kTile samples; thread t owns fixed gradient entries and sums them
// over its CTA's tiles in order; partial[cta][P] and lpart[cta] are then reduced in order.
__global__ void __launch_bounds__(kMThreads)
mlp_grad_kernel(const float* __restrict__ params, int L, float U, const uint32_t* __restrict__ upb,
                const uint32_t* __restrict__ dnb, int64_t dim_dn, const int64_t* __restrict__ idx,
                const double* __restrict__ target, int64_t n, double wscale,
                float* __restrict__ partial, double* __restrict__ lpart) {
  extern __shared__ float smem[];
  const MlpDims d = mlp_dims(L);
  float* sw = smem;                     // P
  float* X = sw + ((d.P + 3) / 4) * 4;  // [kTile][nin]
  float* H1 = X + kTile * kMaxIn;       // [kTile][kH]
  float* H2 = H1 + kTile * kH;          // [kTile][kH]
  float* G2 = H2 + kTile * kH;          // [kTile][kH]
  float* G1 = G2 + kTile * kH;          // [kTile][kH]
  float* DO = G1 + kTile * kH;          // [kTile][2]
  float* H1B = DO + 2 * kTile;          // [kTile][kH] bf16-rounded h1 (input of layer 2)
  __shared__ double lred[kMThreads];
  load_weights(params, d.P, sw);
  const float u8b = bf16r(U * 0.125f);
  // owned gradient entries: W2 (kH*kH), W1 (nin*kH), W3 (2*kH), b1, b2 (kH each), b3 (2)
  constexpr int kOwnW2 = kH * kH / kMThreads;  // 16
  float gW2[kOwnW2];
  constexpr int kOwnW1 = (kMaxIn * kH + kMThreads - 1) / kMThreads;  // 17
  float gW1[kOwnW1];
  float gX = 0.f;   // thread t: W3 entry t (t < 128), b1 (t < 192), b2 (t < 256)
  float gB3 = 0.f;  // threads 0 and 1: b3
  const int nW1 = d.nin * kH;
  const int nW1own = (nW1 + kMThreads - 1) / kMThreads;
#pragma unroll
  for (int q = 0; q < kOwnW2; ++q) gW2[q] = 0.f;
#pragma unroll
  for (int q = 0; q < kOwnW1; ++q) gW1[q] = 0.f;
  double lsum = 0.0;
  const int64_t ntiles = (n + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t s0 = tile * kTile;
    // ---- forward: one thread per (sample, half of the hidden units) for layer 1 and 2
    for (int i = threadIdx.x; i < kTile * d.nin; i += blockDim.x) {
      const int sidx = i / d.nin, f = i - sidx * d.nin;
      const int64_t k = s0 + sidx;
      float v = 0.f;
      if (k < n) {
        const int64_t g = idx[k];
        const int64_t u = g / dim_dn, dd = g - u * dim_dn;
        if (f < L) v = (float)((upb[u] >> f) & 1u);
        else if (f < 2 * L) v = (float)((dnb[dd] >> (f - L)) & 1u);
        else v = u8b;
      }
      X[sidx * kMaxIn + f] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kTile * kH; i += blockDim.x) {
      const int sidx = i / kH, o = i - sidx * kH;
      float s = sw[d.ob1 + o];
      for (int f = 0; f < d.nin; ++f) s = fmaf(X[sidx * kMaxIn + f], sw[d.oW1 + f * kH + o], s);
      const float h = tanhf(s);
      H1[sidx * kH + o] = h;
      H1B[sidx * kH + o] = bf16r(h);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kTile * kH; i += blockDim.x) {
      const int sidx = i / kH, o = i - sidx * kH;
      float s = sw[d.ob2 + o];
      for (int f = 0; f < kH; ++f) s = fmaf(H1B[sidx * kH + f], sw[d.oW2 + f * kH + o], s);
      H2[sidx * kH + o] = tanhf(s);
    }
    __syncthreads();
    // ---- outputs, loss and d(loss)/d(a, z) per sample
    if (threadIdx.x < kTile) {
      const int sidx = threadIdx.x;
      const int64_t k = s0 + sidx;
      float da = 0.f, dz = 0.f;
      if (k < n) {
        float a = sw[d.ob3], z = sw[d.ob3 + 1];
        for (int o = 0; o < kH; ++o) {
          a = fmaf(H2[sidx * kH + o], sw[d.oW3 + 2 * o], a);
          z = fmaf(H2[sidx * kH + o], sw[d.oW3 + 2 * o + 1], z);
        }
        const double psi = target[k];
        if (psi != 0.0) {
          const double w = wscale * psi * psi;
          const double l = log(fabs(psi));
          const double sg = psi >= 0.0 ? 1.0 : -1.0;
          const double diff = (double)a - l;
          const double mz = -sg * (double)z;
          const double sp = mz > 0.0 ? mz + log1p(exp(-mz)) : log1p(exp(mz));
          lsum += w * (diff * diff + sp);
          da = (float)(w * 2.0 * diff / (double)n);
          dz = (float)(w * (-sg) / (1.0 + exp(sg * (double)z)) / (double)n);
        }
      }
      DO[2 * sidx] = da;
      DO[2 * sidx + 1] = dz;
    }
    __syncthreads();
    // ---- backward through layer 2 and 1
    for (int i = threadIdx.x; i < kTile * kH; i += blockDim.x) {
      const int sidx = i / kH, o = i - sidx * kH;
      const float h = H2[sidx * kH + o];
      const float g = fmaf(DO[2 * sidx], sw[d.oW3 + 2 * o], DO[2 * sidx + 1] * sw[d.oW3 + 2 * o + 1]);
      G2[sidx * kH + o] = g * (1.f - h * h);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kTile * kH; i += blockDim.x) {
      const int sidx = i / kH, o = i - sidx * kH;
      float g = 0.f;
      for (int f = 0; f < kH; ++f) g = fmaf(G2[sidx * kH + f], sw[d.oW2 + o * kH + f], g);
      const float h = H1[sidx * kH + o];
      G1[sidx * kH + o] = g * (1.f - h * h);
    }
    __syncthreads();
    // ---- weight gradients owned by this thread (sum over the tile's samples in order)
#pragma unroll
    for (int q = 0; q < kOwnW2; ++q) {
      const int e = threadIdx.x + q * kMThreads;  // W2 entry (i, o)
      const int i = e / kH, o = e - i * kH;
      float acc = 0.f;
      for (int sidx = 0; sidx < kTile; ++sidx) acc = fmaf(H1B[sidx * kH + i], G2[sidx * kH + o], acc);
      gW2[q] += acc;
    }
#pragma unroll
    for (int q = 0; q < kOwnW1; ++q) {
      const int e = threadIdx.x + q * kMThreads;
      if (q < nW1own && e < nW1) {
        const int f = e / kH, o = e - f * kH;
        float acc = 0.f;
        for (int sidx = 0; sidx < kTile; ++sidx) acc = fmaf(X[sidx * kMaxIn + f], G1[sidx * kH + o], acc);
        gW1[q] += acc;
      }
    }
    if (threadIdx.x < 2) {
      float acc = 0.f;
      for (int sidx = 0; sidx < kTile; ++sidx) acc += DO[2 * sidx + threadIdx.x];
      gB3 += acc;
    }
    {
      const int t = threadIdx.x;
      float acc = 0.f;
      if (t < 2 * kH) {  // W3 (o, c)
        const int o = t >> 1, c = t & 1;
        for (int sidx = 0; sidx < kTile; ++sidx) acc = fmaf(H2[sidx * kH + o], DO[2 * sidx + c], acc);
      } else if (t < 3 * kH) {  // b1
        for (int sidx = 0; sidx < kTile; ++sidx) acc += G1[sidx * kH + (t - 2 * kH)];
      } else if (t < 4 * kH) {  // b2
        for (int sidx = 0; sidx < kTile; ++sidx) acc += G2[sidx * kH + (t - 3 * kH)];
      }
      gX += acc;
    }
    __syncthreads();
  }
  float* out = partial + (size_t)blockIdx.x * d.P;
#pragma unroll
  for (int q = 0; q < kOwnW2; ++q) out[d.oW2 + threadIdx.x + q * kMThreads] = gW2[q];
#pragma unroll
  for (int q = 0; q < kOwnW1; ++q) {
    const int e = threadIdx.x + q * kMThreads;
    if (q < nW1own && e < nW1) out[d.oW1 + e] = gW1[q];
  }
  if (threadIdx.x < 2) out[d.ob3 + threadIdx.x] = gB3;
  if (threadIdx.x < 2 * kH) out[d.oW3 + threadIdx.x] = gX;
  else if (threadIdx.x < 3 * kH) out[d.ob1 + threadIdx.x - 2 * kH] = gX;
  else if (threadIdx.x < 4 * kH) out[d.ob2 + threadIdx.x - 3 * kH] = gX;
  lred[threadIdx.x] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < kMThreads; ++i) s += lred[i];
    lpart[blockIdx.x] = s / (double)n;
  }
}

// Sum of the per-CTA partials in CTA order, the mean loss, and optionally an Adam step on
// the master weights.
__global__ void __launch_bounds__(kMThreads)
mlp_reduce_kernel(const float* __restrict__ partial, int ncta, int P, const double* __restrict__ lpart, float* __restrict__ grad, double* __restrict__ loss,
                  float* __restrict__ params, float* __restrict__ m, float* __restrict__ v, int step,
                  float lr, int do_adam) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    float g = 0.f;
    for (int c = 0; c < ncta; ++c) g += partial[(size_t)c * P + i];
    grad[i] = g;
    if (do_adam) {
      const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
      const float mi = b1 * m[i] + (1.f - b1) * g;
      const float vi = b2 * v[i] + (1.f - b2) * g * g;
      m[i] = mi;
      v[i] = vi;
      const float mh = mi / (1.f - powf(b1, (float)step));
      const float vh = vi / (1.f - powf(b2, (float)step));
      params[i] -= lr * mh / (sqrtf(vh) + eps);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int c = 0; c < ncta; ++c) s += lpart[c];
    *loss = s;
  }
}

// Uniform sample of batch indices (SplitMix64 counters) and their target amplitudes.
__global__ void mlp_sample_kernel(uint64_t seed, int64_t dim, int64_t n, const double* __restrict__ psi,
                                  int64_t* __restrict__ idx, double* __restrict__ tgt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + ((uint64_t)k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    const int64_t g = (int64_t)((unsigned __int128)z * (unsigned long long)dim >> 64);
    idx[k] = g;
    tgt[k] = psi[g];
  }
}

// Glorot-uniform initial weights from SplitMix64 counters; biases zero.
__global__ void mlp_init_kernel(int L, uint64_t seed, float* __restrict__ params) {
  const MlpDims d = mlp_dims(L);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.P; i += gridDim.x * blockDim.x) {
    int fan_in = 0, fan_out = 0;
    if (i < d.ob1) fan_in = d.nin, fan_out = kH;
    else if (i >= d.oW2 && i < d.ob2) fan_in = kH, fan_out = kH;
    else if (i >= d.oW3 && i < d.ob3) fan_in = kH, fan_out = 2;
    float v = 0.f;
    if (fan_in) {
      uint64_t z = seed + ((uint64_t)i + 1ull) * 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z = z ^ (z >> 31);
      const double u = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
      v = (float)(u * sqrt(6.0 / (fan_in + fan_out)));
    }
    params[i] = v;
  }
}

}  // namespace ed

using namespace ed;

struct ed_mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  int L = 0;
  MlpDims d{};
  float* params = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  float* partial = nullptr;
  double* lpart = nullptr;
  double* loss = nullptr;
  int64_t* idx = nullptr;
  double* tgt = nullptr;
  int64_t cap = 0;  // batch capacity of idx / tgt
  int ncta = 0;
  int step = 0;
  int* err = nullptr;  // timeout flag of the inference kernel
};

namespace {
size_t grad_smem(const MlpDims& d) {
  return ((size_t)(d.P + 3) / 4 * 4 + (size_t)kTile * kMaxIn + 5 * (size_t)kTile * kH + 2 * kTile) *
         sizeof(float);
}

ed_status mlp_grad(ed_mlp* M, const ed_basis* b, double U, const int64_t* idx, const double* tgt,
                   int64_t n, double wscale, int adam, float lr) {
  cudaStream_t s = M->stream;
  const size_t sm = grad_smem(M->d);
  ED_TRY_CUDA(allow_max_smem(mlp_grad_kernel));
  mlp_grad_kernel<<<M->ncta, kMThreads, sm, s>>>(M->params, M->L, (float)U, b->user_up().bits,
                                                  b->user_dn().bits, b->user_dn().dim, idx, tgt, n,
                                                  wscale, M->partial, M->lpart);
  if (adam) ++M->step;
  mlp_reduce_kernel<<<(M->d.P + kMThreads - 1) / kMThreads, kMThreads, 0, s>>>(
      M->partial, M->ncta, M->d.P, M->lpart, M->grad, M->loss, M->params, M->m,
      M->v, M->step, lr, adam);
  ED_TRY_CUDA(cudaGetLastError());
  return ED_OK;
}
}  // namespace

extern "C" void ed_mlp_destroy(ed_mlp* M) {
  if (!M) return;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != M->device) cudaSetDevice(M->device);
  if (M->stream) cudaStreamSynchronize(M->stream);
  float* fs[] = {M->params, M->m, M->v, M->grad, M->partial};
  for (float* f : fs)
    if (f) cudaFree(f);
  if (M->lpart) cudaFree(M->lpart);
  if (M->loss) cudaFree(M->loss);
  if (M->idx) cudaFree(M->idx);
  if (M->tgt) cudaFree(M->tgt);
  if (M->err) cudaFree(M->err);
  if (prev != M->device) cudaSetDevice(prev);
  delete M;
}

extern "C" ed_status ed_mlp_create(int32_t n_sites, uint64_t seed, void* stream, ed_mlp** out) {
  clear_error();
  ED_CHECK_ARG(out != nullptr, "ed_mlp_create: out is NULL");
  *out = nullptr;
  ED_CHECK_ARG(n_sites >= 1 && n_sites <= kMaxSites, "ed_mlp_create: n_sites outside [1, 32]");
  ed_mlp* M = new ed_mlp();
  cudaGetDevice(&M->device);
  M->stream = (cudaStream_t)stream;
  M->L = n_sites;
  M->d = mlp_dims(n_sites);
  M->ncta = sm_count();
  const size_t P = M->d.P;
  bool ok = cudaMalloc((void**)&M->params, P * 4) == cudaSuccess &&
            cudaMalloc((void**)&M->m, P * 4) == cudaSuccess &&
            cudaMalloc((void**)&M->v, P * 4) == cudaSuccess &&
            cudaMalloc((void**)&M->grad, P * 4) == cudaSuccess &&
            cudaMalloc((void**)&M->partial, (size_t)M->ncta * P * 4) == cudaSuccess &&
            cudaMalloc((void**)&M->lpart, (size_t)M->ncta * 8) == cudaSuccess &&
            cudaMalloc((void**)&M->loss, 8) == cudaSuccess &&
            cudaMalloc((void**)&M->err, sizeof(int)) == cudaSuccess;
  if (!ok) {
    ed_mlp_destroy(M);
    set_error("ed_mlp_create: out of device memory");
    return ED_ERR_OOM;
  }
  mlp_init_kernel<<<(int)((P + 255) / 256), 256, 0, M->stream>>>(n_sites, seed, M->params);
  cudaMemsetAsync(M->m, 0, P * 4, M->stream);
  cudaMemsetAsync(M->v, 0, P * 4, M->stream);
  if (cudaGetLastError() != cudaSuccess) {
    ed_mlp_destroy(M);
    set_error("ed_mlp_create: initialisation failed");
    return ED_ERR_CUDA;
  }
  *out = M;
  return ED_OK;
}

extern "C" ed_status ed_mlp_params(ed_mlp* M, float** params, int64_t* count) {
  clear_error();
  ED_CHECK_ARG(M != nullptr, "ed_mlp_params: NULL handle");
  if (params) *params = M->params;
  if (count) *count = M->d.P;
  return ED_OK;
}

extern "C" ed_status ed_mlp_loss_grad(ed_mlp* M, const ed_basis* b, double U, const int64_t* idx,
                                      const double* target, int64_t n, double weight_scale,
                                      double* loss, const float** grad) {
  clear_error();
  ED_CHECK_ARG(M && b && idx && target && n >= 1, "ed_mlp_loss_grad: bad arguments");
  ED_CHECK_ARG(b->n_sites == M->L, "ed_mlp_loss_grad: basis has %d sites, network %d", b->n_sites, M->L);
  ed_status r = mlp_grad(M, b, U, idx, target, n, weight_scale, 0, 0.f);
  if (r != ED_OK) return r;
  if (loss) {
    ED_TRY_CUDA(cudaMemcpyAsync(loss, M->loss, 8, cudaMemcpyDeviceToHost, M->stream));
    ED_TRY_CUDA(cudaStreamSynchronize(M->stream));
  }
  if (grad) *grad = M->grad;
  return ED_OK;
}

extern "C" ed_status ed_mlp_train_step(ed_mlp* M, const ed_basis* b, double U, const double* psi,
                                       int64_t batch, double lr, uint64_t seed, double* loss) {
  clear_error();
  ED_CHECK_ARG(M && b && psi && batch >= 1 && batch <= (1LL << 24), "ed_mlp_train_step: bad arguments");
  ED_CHECK_ARG(b->n_sites == M->L, "ed_mlp_train_step: basis has %d sites, network %d", b->n_sites, M->L);
  if (batch > M->cap) {
    if (M->idx) cudaFree(M->idx);
    if (M->tgt) cudaFree(M->tgt);
    M->idx = nullptr;
    M->tgt = nullptr;
    M->cap = 0;
    ED_TRY_CUDA(cudaMalloc((void**)&M->idx, batch * 8));
    ED_TRY_CUDA(cudaMalloc((void**)&M->tgt, batch * 8));
    M->cap = batch;
  }
  mlp_sample_kernel<<<sm_count() * 4, 256, 0, M->stream>>>(seed, b->dim, batch, psi, M->idx, M->tgt);
  ED_TRY_CUDA(cudaGetLastError());
  ed_status r = mlp_grad(M, b, U, M->idx, M->tgt, batch, (double)b->dim, 1, (float)lr);
  if (r != ED_OK) return r;
  if (loss) {
    ED_TRY_CUDA(cudaMemcpyAsync(loss, M->loss, 8, cudaMemcpyDeviceToHost, M->stream));
    ED_TRY_CUDA(cudaStreamSynchronize(M->stream));
  }
  return ED_OK;
}

extern "C" ed_status ed_mlp_infer(ed_mlp* M, const ed_basis* b, double U, ed_dtype dtype, void* out) {
  clear_error();
  ED_CHECK_ARG(M && b && out && aligned16(out), "ed_mlp_infer: bad arguments");
  ED_CHECK_ARG(b->n_sites == M->L, "ed_mlp_infer: basis has %d sites, network %d", b->n_sites, M->L);
  const TcLayout ly = tc_layout(M->d.nin);
  const int sm = (int)std::max<uint32_t>(ly.total, (uint32_t)kTcSmemMin);
  const int64_t ntiles = (b->dim + kTcRows - 1) / kTcRows;
  ED_TRY_CUDA(allow_max_smem(mlp_infer_tc_kernel<float>));
  ED_TRY_CUDA(allow_max_smem(mlp_infer_tc_kernel<double>));
  // one wave of resident CTAs: kTcCtasPerSm while the shared memory allows them, else fewer
  int dev = 0, sm_bytes = 0, reserved = 0;
  ED_TRY_CUDA(cudaGetDevice(&dev));
  ED_TRY_CUDA(cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  ED_TRY_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
  const int per_sm = std::max(1, std::min(kTcCtasPerSm, sm_bytes / (sm + reserved)));
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)sm_count() * per_sm);
  ED_TRY_CUDA(cudaMemsetAsync(M->err, 0, sizeof(int), M->stream));
  if (dtype == ED_F32) {
    mlp_infer_tc_kernel<float><<<grid, kTcRows, sm, M->stream>>>(
        M->params, M->L, (float)U, b->user_up().bits, b->user_dn().bits, b->user_dn().dim, b->dim,
        (float*)out, M->err);
  } else {
    mlp_infer_tc_kernel<double><<<grid, kTcRows, sm, M->stream>>>(
        M->params, M->L, (float)U, b->user_up().bits, b->user_dn().bits, b->user_dn().dim, b->dim,
        (double*)out, M->err);
  }
  ED_TRY_CUDA(cudaGetLastError());
  int h = 0;
  ED_TRY_CUDA(cudaMemcpyAsync(&h, M->err, sizeof(int), cudaMemcpyDeviceToHost, M->stream));
  ED_TRY_CUDA(cudaStreamSynchronize(M->stream));
  if (h) {
    set_error("ed_mlp_infer: a tensor-core completion wait ran out");
    return ED_ERR_TIMEOUT;
  }
  return ED_OK;
}

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
// Training: samples drawn uniformly from the basis with weight dim * psi^2; loss per sample
// (a - log|psi|)^2 + log(1 + exp(-sign(psi) z)); deterministic per-CTA gradient partials
// reduced in a fixed order.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "ed_internal.cuh"

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

// Rounded weights into shared memory (sw has P floats).
__device__ __forceinline__ void load_weights(const float* __restrict__ params, int P, float* sw) {
  for (int i = threadIdx.x; i < P; i += blockDim.x) sw[i] = bf16r(params[i]);
  __syncthreads();
}

// ------------------------------------------------------------------ inference
// BF16 tensor-core products (mma.sync m16n8k16, FP32 accumulation): a warp evaluates 16
// basis states at a time. Thread (g = lane/4, q = lane%4) holds rows g and g+8 of every
// fragment; the first layer's accumulator fragments are, after tanh and rounding, exactly
// the A fragments of the second layer (its K index is the first layer's N index), so the
// activations never leave registers.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

constexpr int kMaxKT1 = (kMaxIn + 15) / 16;  // k-tiles of the first layer

// B fragments of a K x 64 weight block (row-major W[k][n], rows >= K are zero) into shared
// memory: frag[(kt * 8 + nt) * 32 + lane] = (W[k0..k0+1][n], W[k0+8..k0+9][n]) packed,
// k0 = kt*16 + 2q, n = nt*8 + g.
__device__ void build_frags(const float* W, int K, int KT, uint2* frag) {
  for (int i = threadIdx.x; i < KT * 8 * 32; i += blockDim.x) {
    const int lane = i & 31, nt = (i >> 5) & 7, kt = i >> 8;
    const int g = lane >> 2, q = lane & 3;
    const int n = nt * 8 + g, k0 = kt * 16 + 2 * q;
    auto w = [&](int k) { return k < K ? W[k * kH + n] : 0.f; };
    frag[i] = make_uint2(pack_bf16(w(k0), w(k0 + 1)), pack_bf16(w(k0 + 8), w(k0 + 9)));
  }
}

template <typename T>
__global__ void __launch_bounds__(kMThreads)
mlp_infer_kernel(const float* __restrict__ params, int L, float U, const uint32_t* __restrict__ upb,
                 const uint32_t* __restrict__ dnb, int64_t dim_dn, int64_t dim, T* __restrict__ out) {
  __shared__ uint2 f1[kMaxKT1 * 8 * 32];
  __shared__ uint2 f2[4 * 8 * 32];
  __shared__ float sb1[kH], sb2[kH], sW3[2 * kH], sb3[2];
  extern __shared__ float sw[];
  const MlpDims d = mlp_dims(L);
  const int KT1 = (d.nin + 15) / 16;
  load_weights(params, d.P, sw);  // rounded weights
  build_frags(sw + d.oW1, d.nin, KT1, f1);
  build_frags(sw + d.oW2, kH, 4, f2);
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    sb1[i] = sw[d.ob1 + i];
    sb2[i] = sw[d.ob2 + i];
    sW3[2 * i] = sw[d.oW3 + 2 * i];
    sW3[2 * i + 1] = sw[d.oW3 + 2 * i + 1];
  }
  if (threadIdx.x < 2) sb3[threadIdx.x] = sw[d.ob3 + threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const float u8 = bf16r(U * 0.125f);
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (int64_t base = wid * 16; base < dim; base += warps * 16) {
    const int64_t e0 = base + g, e1 = base + g + 8;
    uint32_t ub0 = 0, db0 = 0, ub1 = 0, db1 = 0;
    if (e0 < dim) {
      const int64_t u = e0 / dim_dn;
      ub0 = upb[u];
      db0 = dnb[e0 - u * dim_dn];
    }
    if (e1 < dim) {
      const int64_t u = e1 / dim_dn;
      ub1 = upb[u];
      db1 = dnb[e1 - u * dim_dn];
    }
    auto feat = [&](uint32_t ub, uint32_t db, int f) -> float {
      if (f < L) return (float)((ub >> f) & 1u);
      if (f < 2 * L) return (float)((db >> (f - L)) & 1u);
      return f == 2 * L ? u8 : 0.f;
    };
    // ---- layer 1: acc[nt] = b1 + x W1 over KT1 k-tiles
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float c0 = sb1[nt * 8 + 2 * q], c1 = sb1[nt * 8 + 2 * q + 1];
      acc[nt][0] = c0;
      acc[nt][1] = c1;
      acc[nt][2] = c0;
      acc[nt][3] = c1;
    }
    for (int kt = 0; kt < KT1; ++kt) {
      const int c = kt * 16 + 2 * q;
      uint32_t A[4];
      A[0] = pack_bf16(feat(ub0, db0, c), feat(ub0, db0, c + 1));
      A[1] = pack_bf16(feat(ub1, db1, c), feat(ub1, db1, c + 1));
      A[2] = pack_bf16(feat(ub0, db0, c + 8), feat(ub0, db0, c + 9));
      A[3] = pack_bf16(feat(ub1, db1, c + 8), feat(ub1, db1, c + 9));
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) mma_bf16(acc[nt], A, f1[(kt * 8 + nt) * 32 + lane]);
    }
    // ---- layer 2: A fragments from tanh(layer 1), acc2 = b2 + h1 W2
    uint32_t A2[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      A2[kt][0] = pack_bf16(tanhf(acc[2 * kt][0]), tanhf(acc[2 * kt][1]));
      A2[kt][1] = pack_bf16(tanhf(acc[2 * kt][2]), tanhf(acc[2 * kt][3]));
      A2[kt][2] = pack_bf16(tanhf(acc[2 * kt + 1][0]), tanhf(acc[2 * kt + 1][1]));
      A2[kt][3] = pack_bf16(tanhf(acc[2 * kt + 1][2]), tanhf(acc[2 * kt + 1][3]));
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float c0 = sb2[nt * 8 + 2 * q], c1 = sb2[nt * 8 + 2 * q + 1];
      acc[nt][0] = c0;
      acc[nt][1] = c1;
      acc[nt][2] = c0;
      acc[nt][3] = c1;
    }
#pragma unroll
    for (int kt = 0; kt < 4; ++kt)
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) mma_bf16(acc[nt], A2[kt], f2[(kt * 8 + nt) * 32 + lane]);
    // ---- layer 3: partial dot products over this thread's 16 hidden units, then the 4 lanes
    float a0 = 0.f, z0 = 0.f, a1 = 0.f, z1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int c = nt * 8 + 2 * q;
      const float h00 = tanhf(acc[nt][0]), h01 = tanhf(acc[nt][1]);
      const float h10 = tanhf(acc[nt][2]), h11 = tanhf(acc[nt][3]);
      a0 = fmaf(h00, sW3[2 * c], fmaf(h01, sW3[2 * c + 2], a0));
      z0 = fmaf(h00, sW3[2 * c + 1], fmaf(h01, sW3[2 * c + 3], z0));
      a1 = fmaf(h10, sW3[2 * c], fmaf(h11, sW3[2 * c + 2], a1));
      z1 = fmaf(h10, sW3[2 * c + 1], fmaf(h11, sW3[2 * c + 3], z1));
    }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      z0 += __shfl_xor_sync(0xffffffffu, z0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
      z1 += __shfl_xor_sync(0xffffffffu, z1, o);
    }
    if (q == 0) {
      a0 += sb3[0];
      z0 += sb3[1];
      a1 += sb3[0];
      z1 += sb3[1];
      if (e0 < dim) {
        const float v = expf(a0);
        out[e0] = (T)(z0 >= 0.f ? v : -v);
      }
      if (e1 < dim) {
        const float v = expf(a1);
        out[e1] = (T)(z1 >= 0.f ? v : -v);
      }
    }
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
  ED_TRY_CUDA(cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
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
            cudaMalloc((void**)&M->loss, 8) == cudaSuccess;
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
  const size_t sm = (size_t)M->d.P * sizeof(float);
  const int grid = sm_count() * 8;
  if (dtype == ED_F32) {
    ED_TRY_CUDA(cudaFuncSetAttribute(mlp_infer_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    mlp_infer_kernel<float><<<grid, kMThreads, sm, M->stream>>>(M->params, M->L, (float)U,
                                                                b->user_up().bits, b->user_dn().bits,
                                                                b->user_dn().dim, b->dim, (float*)out);
  } else {
    ED_TRY_CUDA(cudaFuncSetAttribute(mlp_infer_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    mlp_infer_kernel<double><<<grid, kMThreads, sm, M->stream>>>(M->params, M->L, (float)U,
                                                                 b->user_up().bits, b->user_dn().bits,
                                                                 b->user_dn().dim, b->dim, (double*)out);
  }
  ED_TRY_CUDA(cudaGetLastError());
  return ED_OK;
}

// Double occupancy of a state vector: D_i = <psi| n_i,up n_i,dn |psi> / <psi|psi> (the
// on-site operator of the interaction term added to Sec. 1 Eq. 1) and D = sum_i D_i, which
// equals dE0/dU for a normalised non-degenerate ground state (Hellmann-Feynman).
//
// One pass over psi (FP64, basis order u * dim_dn + d): each thread accumulates psi^2, the
// per-site sums over the doubly occupied sites of its elements (m = up_u & dn_d) and
// psi^2 popc(m); CTAs write partials that one CTA sums in a fixed order.
#include "ed_internal.cuh"

namespace ed {

constexpr int kObsThreads = 256;
constexpr int kObsSums = 34;  // norm^2, total, 32 sites

__global__ void __launch_bounds__(kObsThreads)
obs_partials_kernel(const double* __restrict__ psi, const uint32_t* __restrict__ up,
                    const uint32_t* __restrict__ dn, int64_t dim_dn, int64_t dim, int n_sites,
                    double* __restrict__ part) {
  __shared__ double red[33];
  double nrm = 0.0, tot = 0.0, site[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) site[i] = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < dim;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = e / dim_dn, d = e - u * dim_dn;
    const double v = psi[e];
    const double p2 = v * v;
    const uint32_t m = up[u] & dn[d];
    nrm += p2;
    tot = fma(p2, (double)__popc(m), tot);
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if ((m >> i) & 1u) site[i] += p2;
  }
  const double nr = block_sum(nrm, red);
  __syncthreads();
  const double tr = block_sum(tot, red);
  __syncthreads();
  if (threadIdx.x == 0) {
    part[(int64_t)blockIdx.x * kObsSums + 0] = nr;
    part[(int64_t)blockIdx.x * kObsSums + 1] = tr;
  }
#pragma unroll
  for (int i = 0; i < 32; ++i) {  // constant indices keep site[] in registers
    if (i < n_sites) {
      const double si = block_sum(site[i], red);
      __syncthreads();
      if (threadIdx.x == 0) part[(int64_t)blockIdx.x * kObsSums + 2 + i] = si;
    }
  }
}

// One CTA: column sums of the partials in CTA order.
__global__ void __launch_bounds__(kObsThreads)
obs_final_kernel(const double* __restrict__ part, int nparts, int nsums, double* __restrict__ out) {
  __shared__ double red[33];
  for (int k = 0; k < nsums; ++k) {
    double v = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += part[(int64_t)i * kObsSums + k];
    v = block_sum(v, red);
    __syncthreads();
    if (threadIdx.x == 0) out[k] = v;
  }
}

}  // namespace ed

using namespace ed;

extern "C" ed_status ed_double_occupancy(const ed_basis* b, const double* psi, void* stream,
                                         double* D_total, double* D_site) {
  clear_error();
  ED_CHECK_ARG(b && psi && D_total, "ed_double_occupancy: NULL argument");
  ED_CHECK_ARG(aligned16(psi), "ed_double_occupancy: psi must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const int nsums = 2 + b->n_sites;
  int64_t g64 = (b->dim + kObsThreads - 1) / kObsThreads;
  const int64_t cap = (int64_t)sm_count() * 4;
  const int grid = (int)(g64 < 1 ? 1 : (g64 < cap ? g64 : cap));
  double* part = nullptr;
  ED_TRY_CUDA(cudaMallocAsync((void**)&part, ((size_t)grid * kObsSums + kObsSums) * sizeof(double), s));
  double* out = part + (size_t)grid * kObsSums;
  obs_partials_kernel<<<grid, kObsThreads, 0, s>>>(psi, b->up.bits, b->dn.bits, b->dn.dim, b->dim,
                                                   b->n_sites, part);
  obs_final_kernel<<<1, kObsThreads, 0, s>>>(part, grid, nsums, out);
  double h[kObsSums] = {0.0};
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, nsums * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(part, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error("ed_double_occupancy: %s", cudaGetErrorString(e));
    return ED_ERR_CUDA;
  }
  ED_CHECK_ARG(h[0] > 0.0, "ed_double_occupancy: psi is the zero vector");
  *D_total = h[1] / h[0];
  if (D_site)
    for (int i = 0; i < b->n_sites; ++i) D_site[i] = h[2 + i] / h[0];
  return ED_OK;
}

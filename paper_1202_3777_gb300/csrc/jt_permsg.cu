// The paper's own message kernel (Algorithm 1), for comparison with the
// fused persistent kernel: one launch per message, one thread per separator
// entry j, which gathers the clique entries mapped to j through a
// precomputed index-mapping table mu (Sec. 3.2, Fig. 3), marginalises
// (Eq. 2), forms the ratio with 0/0 := 0 (Eq. 3) and scatters it into the
// neighbour (Eq. 1).  The mapping tables are laid out as the paper compares
// them (Sec. 4.5, Fig. 8): naive, every separator entry's list contiguous,
// or interleaved, the m-th elements of all lists adjacent.  Messages are
// split in two launches (marginalise, then ratio and scatter) so that a
// collect message can be normalised by its total before it is applied;
// sums are kept in double.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "jt_kernels.h"

namespace jt {
namespace {

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
  return t;  // valid in thread 0
}

__device__ __forceinline__ int32_t mu_at(const int32_t* mu, int32_t j, int32_t m, int32_t L, int32_t S,
                                         int interleaved) {
  return interleaved ? mu[(int64_t)m * S + j] : mu[(int64_t)j * L + m];
}

// snew[j] = sum_m phi[mu(j, m)]; *sigma += sum_j snew[j].
template <typename T>
__global__ void __launch_bounds__(256) k_msg_marg(const T* phi, const int32_t* mu, int32_t L, int32_t S,
                                                  int interleaved, double* snew, double* sigma) {
  const int32_t j = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  double v = 0.0;
  if (j < S) {
    for (int32_t m = 0; m < L; ++m) v += (double)phi[mu_at(mu, j, m, L, S, interleaved)];
    snew[j] = v;
  }
  const double t = block_sum(v);
  if (threadIdx.x == 0 && t != 0.0) atomicAdd(sigma, t);
}

// n = snew[j] (divided by *sigma when normalising); r = n / sold[j], 0 if
// sold[j] = 0; sold[j] = n; phi[mu(j, m)] *= r for every m.
template <typename T>
__global__ void __launch_bounds__(256) k_msg_scatter(T* phi, const int32_t* mu, int32_t L, int32_t S,
                                                     int interleaved, const double* snew, T* sold,
                                                     const double* sigma, int normalise) {
  const int32_t j = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (j >= S) return;
  double n = snew[j];
  if (normalise) {
    const double sg = *sigma;
    n = sg > 0.0 ? n / sg : 0.0;
  }
  const double o = (double)sold[j];
  const T r = (T)(o != 0.0 ? n / o : 0.0);
  sold[j] = (T)n;
  for (int32_t m = 0; m < L; ++m) phi[mu_at(mu, j, m, L, S, interleaved)] *= r;
}

// Zero the entries of one clique that contradict the evidence: obs holds
// (stride, cardinality, state) of each observed variable of the clique.
template <typename T>
__global__ void __launch_bounds__(256) k_clique_evidence(T* phi, int64_t n, const int4* obs, int n_obs) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    bool keep = true;
    for (int i = 0; i < n_obs; ++i) {
      const int4 o = obs[i];
      if ((int)((x / o.x) % o.y) != o.z) keep = false;
    }
    if (!keep) phi[x] = T(0);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_table_sum(const T* phi, int64_t n, double* out) {
  double v = 0.0;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
    v += (double)phi[x];
  const double t = block_sum(v);
  if (threadIdx.x == 0 && t != 0.0) atomicAdd(out, t);
}

template <typename T>
__global__ void __launch_bounds__(256) k_table_scale(T* phi, int64_t n, const double* total) {
  const double z = *total;
  const T f = (T)(z > 0.0 ? 1.0 / z : 0.0);
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
    phi[x] *= f;
}

// The stage totals the finalisation reads: sums[c] = sigma_c * |S_c| for
// every collect message (so that log sums[c] - log |S_c| = log sigma_c) and
// sums[n_cliques] = the root's total.
__global__ void k_pack_totals(const double* sigma, const int32_t* sep_size, int nc, const double* root_total,
                              double* sums) {
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    if (c >= 1) sums[c] = sigma[c] * (double)sep_size[c];
    if (c == 0) sums[nc] = *root_total;
  }
}

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

}  // namespace

template <typename T>
cudaError_t launch_msg_marg(const T* phi, const int32_t* mu, int32_t L, int32_t S, int interleaved, double* snew,
                            double* sigma, cudaStream_t s) {
  k_msg_marg<T><<<(S + 255) / 256, 256, 0, s>>>(phi, mu, L, S, interleaved, snew, sigma);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_msg_scatter(T* phi, const int32_t* mu, int32_t L, int32_t S, int interleaved,
                               const double* snew, T* sold, const double* sigma, int normalise, cudaStream_t s) {
  k_msg_scatter<T><<<(S + 255) / 256, 256, 0, s>>>(phi, mu, L, S, interleaved, snew, sold, sigma, normalise);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_clique_evidence(T* phi, int64_t n, const int4* obs, int n_obs, cudaStream_t s) {
  if (n_obs == 0 || n == 0) return cudaSuccess;
  k_clique_evidence<T><<<grid_for(n), 256, 0, s>>>(phi, n, obs, n_obs);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_table_normalise(T* phi, int64_t n, double* total, cudaStream_t s) {
  k_table_sum<T><<<grid_for(n), 256, 0, s>>>(phi, n, total);
  k_table_scale<T><<<grid_for(n), 256, 0, s>>>(phi, n, total);
  return cudaGetLastError();
}

cudaError_t launch_pack_totals(const double* sigma, const int32_t* sep_size, int nc, const double* root_total,
                               double* sums, cudaStream_t s) {
  k_pack_totals<<<1, 256, 0, s>>>(sigma, sep_size, nc, root_total, sums);
  return cudaGetLastError();
}

template cudaError_t launch_msg_marg<float>(const float*, const int32_t*, int32_t, int32_t, int, double*, double*,
                                            cudaStream_t);
template cudaError_t launch_msg_marg<double>(const double*, const int32_t*, int32_t, int32_t, int, double*, double*,
                                             cudaStream_t);
template cudaError_t launch_msg_scatter<float>(float*, const int32_t*, int32_t, int32_t, int, const double*, float*,
                                               const double*, int, cudaStream_t);
template cudaError_t launch_msg_scatter<double>(double*, const int32_t*, int32_t, int32_t, int, const double*,
                                                double*, const double*, int, cudaStream_t);
template cudaError_t launch_clique_evidence<float>(float*, int64_t, const int4*, int, cudaStream_t);
template cudaError_t launch_clique_evidence<double>(double*, int64_t, const int4*, int, cudaStream_t);
template cudaError_t launch_table_normalise<float>(float*, int64_t, double*, cudaStream_t);
template cudaError_t launch_table_normalise<double>(double*, int64_t, double*, cudaStream_t);

}  // namespace jt

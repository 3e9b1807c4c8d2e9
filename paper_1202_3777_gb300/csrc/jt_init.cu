// Clique tables from the conditional probability tables of a Bayesian
// network: the Initialization step of Algorithm 4 (Sec. 3.3).  Every clique
// table becomes the product of the CPTs assigned to it (one where none is),
// written straight into the resident permuted layout, so a network's tables
// go from host CPTs to a propagatable tree without a host-side pass over the
// clique entries.
//
// One thread per clique entry.  The entry's flat index in the permuted
// table decodes into the state of each clique variable (row-major over the
// permuted order); a CPT's entry is the dot product of its family's states
// with the CPT's strides.  Per CPT only its family's positions are decoded
// (a compact term list), with shifts and masks when every cardinality of
// the clique is a power of two and multiply-shift divisions otherwise.  Work is cut into chunks of one clique each
// so that a grid of a few CTAs per SM streams every table once; the writes
// are coalesced and the CPTs (a few KB per clique) stay in L1/L2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "jt_init.h"

namespace jt {
namespace {

__device__ __forceinline__ uint32_t udiv(uint32_t n, UDiv d) {
  const uint32_t t = __umulhi(d.mul, n);
  return (t + ((n - t) >> d.sh1)) >> d.sh2;
}

// The entries [start, end) of one clique: each thread takes kInitPerThread
// of them, blockDim apart (so every store instruction of a warp covers
// consecutive entries), and runs the factor and term loops once for all of
// them.  `cv` holds the clique's CPTs (shared or global memory).
template <typename T>
__device__ __forceinline__ void init_range(T* out, uint32_t start, uint32_t end, const InitClique& q,
                                           const InitFactor* factors, const InitTerm* terms, const T* cv) {
  constexpr int J = kInitPerThread;
  for (uint32_t e0 = start + threadIdx.x; e0 < end; e0 += J * blockDim.x) {
    T v[J];
#pragma unroll
    for (int j = 0; j < J; ++j) v[j] = T(1);
    for (int32_t f = q.f0; f < q.f0 + q.nf; ++f) {
      const InitFactor F = factors[f];
      int32_t idx[J];
#pragma unroll
      for (int j = 0; j < J; ++j) idx[j] = 0;
      for (int32_t t = F.t0; t < F.t0 + F.nt; ++t) {
        const InitTerm m = terms[t];
        if (q.pow2) {
#pragma unroll
          for (int j = 0; j < J; ++j)
            idx[j] += (int32_t)(((e0 + j * blockDim.x) >> m.shift) & (uint32_t)(m.card - 1)) * m.fstride;
        } else {
#pragma unroll
          for (int j = 0; j < J; ++j) {
            const uint32_t q1 = udiv(e0 + j * blockDim.x, m.pdiv);
            const uint32_t q2 = udiv(q1, m.cdiv);
            idx[j] += (int32_t)(q1 - q2 * (uint32_t)m.card) * m.fstride;
          }
        }
      }
      // every idx is a valid CPT index (each decoded state is below its
      // cardinality), but only entries of the range are read and written
      const T* tab = cv + F.val_off;
#pragma unroll
      for (int j = 0; j < J; ++j)
        if (e0 + j * blockDim.x < end) v[j] *= tab[idx[j]];
    }
#pragma unroll
    for (int j = 0; j < J; ++j)
      if (e0 + j * blockDim.x < end) out[e0 + j * blockDim.x] = v[j];
  }
}

// A CTA walks items; when an item's clique changes and its CPTs fit, they
// are copied to shared memory first, so the per-entry gathers hit shared
// memory rather than L1 lines.
template <typename T>
__global__ void __launch_bounds__(256) k_init_cliques(T* base, const InitItem* items, int32_t n_items,
                                                      const InitClique* cliques, const InitFactor* factors,
                                                      const InitTerm* terms, const T* vals) {
  extern __shared__ __align__(16) unsigned char init_smem[];
  T* s_vals = reinterpret_cast<T*>(init_smem);
  constexpr int32_t cap = kInitSmemBytes / (int32_t)sizeof(T);
  int32_t staged_clique = -1;
  for (int32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const InitItem w = items[it];
    const InitClique q = cliques[w.clique];
    const uint32_t start = (uint32_t)w.start;
    const uint32_t end = (uint32_t)min(w.start + kInitChunk, q.n);
    if (q.nvals <= cap) {
      if (w.clique != staged_clique) {  // uniform over the CTA
        __syncthreads();                // the previous item's gathers are done
        for (int32_t i = threadIdx.x; i < q.nvals; i += blockDim.x) s_vals[i] = vals[q.vals_off + i];
        __syncthreads();
        staged_clique = w.clique;
      }
      init_range<T>(base + q.base_off, start, end, q, factors, terms, s_vals);
    } else {
      init_range<T>(base + q.base_off, start, end, q, factors, terms, vals + q.vals_off);
    }
  }
}

// out[i] = table[permuted offset of listed index i], as double.
template <typename T>
__global__ void __launch_bounds__(256) k_table_unpermute(const T* table, CliqueOut co, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < co.n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i, src = 0;
    for (int j = co.k - 1; j >= 0; --j) {
      const int64_t d = r % co.lcard[j];
      r /= co.lcard[j];
      src += d * co.pst[j];
    }
    out[i] = (double)table[src];
  }
}

// One thread per padded entry, a clique per grid row; the digits of the
// padded layout are bit fields, so the decode is shifts and masks.
__global__ void __launch_bounds__(256) k_pad_tables(const float* __restrict__ base, float* __restrict__ pad,
                                                    const int4* __restrict__ digits,
                                                    const PadClique* __restrict__ cliques, int32_t n_cliques) {
  for (int32_t c = blockIdx.y; c < n_cliques; c += gridDim.y) {
    const PadClique q = cliques[c];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < q.n_pad;
         e += (int64_t)gridDim.x * blockDim.x) {
      int64_t src = 0;
      bool hole = false;
      for (int i = 0; i < q.k; ++i) {
        const int4 g = digits[q.d0 + i];
        const int32_t d = (int32_t)((e >> g.x) & ((1ll << g.y) - 1));
        hole |= d >= g.z;
        src += (int64_t)d * g.w;
      }
      pad[q.off_pad + e] = hole ? 0.f : base[q.off + src];
    }
  }
}

}  // namespace

cudaError_t launch_pad_tables(const float* base, float* pad, const int4* digits, const PadClique* cliques,
                              int32_t n_cliques, int64_t max_pad, cudaStream_t s) {
  if (n_cliques == 0 || max_pad == 0) return cudaSuccess;
  const dim3 grid((unsigned)std::min<int64_t>(256, (max_pad + 255) / 256), (unsigned)std::min(n_cliques, 4096));
  k_pad_tables<<<grid, 256, 0, s>>>(base, pad, digits, cliques, n_cliques);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_cliques(T* base, const InitItem* items, int32_t n_items, const InitClique* cliques,
                                const InitFactor* factors, const InitTerm* terms, const T* vals, int n_sm,
                                cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  // one wave of resident CTAs, each walking its share of the items
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_init_cliques<T>, 256, kInitSmemBytes);
  if (e != cudaSuccess) return e;
  const int grid = std::min<int>(n_items, std::max(1, n_sm) * std::max(1, per_sm));
  k_init_cliques<T><<<grid, 256, kInitSmemBytes, s>>>(base, items, n_items, cliques, factors, terms, vals);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_table_unpermute(const T* table, const CliqueOut& co, double* out_dev, cudaStream_t s) {
  if (co.n == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>(1024, (co.n + 255) / 256);
  k_table_unpermute<T><<<blocks, 256, 0, s>>>(table, co, out_dev);
  return cudaGetLastError();
}

template cudaError_t launch_init_cliques<float>(float*, const InitItem*, int32_t, const InitClique*,
                                                const InitFactor*, const InitTerm*, const float*, int, cudaStream_t);
template cudaError_t launch_init_cliques<double>(double*, const InitItem*, int32_t, const InitClique*,
                                                 const InitFactor*, const InitTerm*, const double*, int,
                                                 cudaStream_t);
template cudaError_t launch_table_unpermute<float>(const float*, const CliqueOut&, double*, cudaStream_t);
template cudaError_t launch_table_unpermute<double>(const double*, const CliqueOut&, double*, cudaStream_t);

}  // namespace jt

// Launch interface of the message kernels (used by the C ABI layer).
#pragma once

#include <cuda_runtime.h>

#include "jt_internal.h"

namespace jt {

// Per-level shared-memory plan, computed on the host and used identically by
// the kernel to carve its dynamic shared memory.
struct SmemPlan {
  int32_t cb;                    // evidence cases handled by one CTA
  int32_t n_child, n_field;      // maxima over the level's cliques
  int32_t n_home, k;
  int32_t tabs;                  // per case: entries of the table region (per-clique residency,
                                 // see DevClique.sm_*)
  int32_t win;                   // per case: collect window of parent-separator entries
  int32_t elem;                  // sizeof(T)
  int32_t stages;                // bulk-copy ring: number of chunk buffers
  int32_t chunk;                 // entries per chunk (= threads x vector width)
  int32_t rowmax;                // per case: rows of one slice (row sums, row factors)
  int32_t pad;
};

struct SmemLayout {
  int32_t off_ch, off_fld, off_hm, off_pos, off_obs, off_nobs;
  int32_t off_facp, off_outp, off_rhop, off_houtp, off_jntp;
  int32_t off_tabs, off_win, off_red, off_bar, off_rsum, off_gsm, off_buf;
  int32_t bytes;

  __host__ __device__ static int32_t a16(int32_t x) { return (x + 15) & ~15; }

  __host__ __device__ explicit SmemLayout(const SmemPlan& s) {
    int32_t o = 0;
    off_ch = o;    o = a16(o + s.n_child * (int32_t)sizeof(DevChild));
    off_fld = o;   o = a16(o + s.n_field * (int32_t)sizeof(DevField));
    off_hm = o;    o = a16(o + s.n_home * (int32_t)sizeof(DevHome));
    off_pos = o;   o = a16(o + s.k * (int32_t)sizeof(DevPos));
    off_obs = o;   o = a16(o + 2 * s.cb * s.k * 8);      // row and column observations
    off_nobs = o;  o = a16(o + 2 * s.cb * 4);
    off_facp = o;  o = a16(o + s.cb * s.n_child * 8);
    off_outp = o;  o = a16(o + s.cb * s.n_child * 8);
    off_rhop = o;  o = a16(o + s.cb * 8);
    off_houtp = o; o = a16(o + s.cb * 8);
    off_jntp = o;  o = a16(o + s.cb * 8);
    off_tabs = o;  o = a16(o + s.cb * s.tabs * s.elem);
    off_win = o;   o = a16(o + s.cb * s.win * s.elem);
    off_red = o;   o = a16(o + 80 * 8);
    off_bar = o;   o = a16(o + 2 * s.stages * 8);   // full and empty barriers
    off_rsum = o;  o = a16(o + s.cb * s.rowmax * s.elem);
    off_gsm = o;   o = a16(o + s.cb * s.rowmax * s.elem);
    o = (o + 127) & ~127;
    off_buf = o;   o += s.stages * s.chunk * s.elem;
    bytes = o;
  }
};

// Cliques whose rows are short enough to be processed inline while streaming
// (the kernel's stream_inline): power-of-two cardinalities, and either no
// private variables with a vector-aligned fastest digit, or vector-aligned
// rows of at most 32 vectors.
__host__ __device__ inline bool inline_rows(const DevClique& c, int vec) {
  if (!c.pow2) return false;
  if (c.P == 1) return c.card_last % vec == 0;
  return c.P % vec == 0 && c.P <= 32 * vec;
}

// Enqueue a whole propagation (collect and distribute of every clique for
// the case range of `a`) as one persistent launch of `grid` CTAs on `s`.
template <typename T>
cudaError_t launch_propagate(const LevelArgs<T>& a, const SmemPlan& sp, int grid, cudaStream_t s);

// Resident CTAs per SM of the propagation kernel for a shared-memory plan.
int32_t propagate_occupancy(int elem, int cb, int bytes);

// Enqueue the finalisation (log Z and normalised marginals) for a case range.
template <typename T>
cudaError_t launch_finalize(const FinalArgs<T>& a, cudaStream_t s);

// Normalised calibrated clique in the caller's listed order.
struct CliqueOut {
  int32_t n, k;
  int32_t lcard[32];             // listed cardinalities
  int32_t pst[32];               // permuted stride of each listed position
};
template <typename T>
cudaError_t launch_get_clique(const T* calib_clique, const CliqueOut& co, double* out_dev,
                              double* sum_dev, cudaStream_t s);

// Maximum dynamic shared memory per CTA the kernels may use on this device.
int32_t smem_budget(int device);

// Consumer threads per CTA of the propagation kernel (plus one producer warp).
constexpr int kLevelThreads = 512;

}  // namespace jt

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
  int32_t n_home, n_src, k;
  int32_t fac;                   // per case: smem entries for child factors (0: read from global)
  int32_t rho;                   // per case: smem entries for the parent ratio (distribute)
  int32_t out;                   // per case: smem entries for outputs (0: accumulate in global)
  int32_t srcacc;                // per case: smem entries for separator-read marginals
  int32_t fac_global, out_global;
  int32_t elem;                  // sizeof(T)
};

struct SmemLayout {
  int32_t off_ch, off_fld, off_hm, off_src, off_pos, off_obs, off_nobs;
  int32_t off_facp, off_outp, off_scale, off_houtp, off_rho, off_fac, off_out, off_srcacc, off_red;
  int32_t bytes;

  __host__ __device__ static int32_t a16(int32_t x) { return (x + 15) & ~15; }

  __host__ __device__ explicit SmemLayout(const SmemPlan& s) {
    int32_t o = 0;
    off_ch = o;    o = a16(o + s.n_child * (int32_t)sizeof(DevChild));
    off_fld = o;   o = a16(o + s.n_field * (int32_t)sizeof(DevField));
    off_hm = o;    o = a16(o + s.n_home * (int32_t)sizeof(DevHome));
    off_src = o;   o = a16(o + s.n_src * (int32_t)sizeof(DevSrc));
    off_pos = o;   o = a16(o + s.k * (int32_t)sizeof(DevPos));
    off_obs = o;   o = a16(o + s.cb * s.k * 8);
    off_nobs = o;  o = a16(o + s.cb * 4);
    off_facp = o;  o = a16(o + s.cb * s.n_child * 8);
    off_outp = o;  o = a16(o + s.cb * s.n_child * 8);
    off_scale = o; o = a16(o + s.cb * s.n_child * s.elem);
    off_houtp = o; o = a16(o + s.cb * 8);
    off_rho = o;   o = a16(o + s.cb * s.rho * s.elem);
    off_fac = o;   o = a16(o + s.cb * s.fac * s.elem);
    off_out = o;   o = a16(o + s.cb * s.out * s.elem);
    off_srcacc = o; o = a16(o + s.cb * s.srcacc * s.elem);
    off_red = o;   o = a16(o + 64 * 8);
    bytes = o;
  }
};

struct LaunchLevel {
  bool collect;
  int32_t n_work;                // CTAs along x
  int32_t n_caseblk;             // CTAs along y
  const DevWork* work;           // device
  SmemPlan sp;
  int32_t pow2_mode;             // 1: every clique of the level is all powers of two
  int32_t vec_mode;              // 1: every clique's fastest cardinality is a multiple of the vector width
};

// Enqueue one level pass (collect or distribute) on `s`.
template <typename T>
cudaError_t launch_level(const LevelArgs<T>& a, const LaunchLevel& L, cudaStream_t s);

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

}  // namespace jt

// Device-side initialisation of the clique tables from the conditional
// probability tables of a Bayesian network (the Initialization step of
// Algorithm 4): descriptor layout and launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "jt_internal.h"
#include "jt_kernels.h"

namespace jt {

// Initialisation of the clique tables from CPTs (Algorithm 4): one item is
// up to kInitChunk consecutive entries of one clique; a clique lists its
// factors [f0, f0 + nf) in ascending CPT order; a factor lists the terms
// [t0, t0 + nt) of its family variables.  A term decodes one variable's
// state from a flat clique index e as (e / pstride) % card and weighs it by
// the variable's stride in the CPT.  When every cardinality of the clique
// is a power of two the decode is (e >> shift) & (card - 1); otherwise both
// divisions are multiply-and-shift by the invariant divisor (pdiv for
// pstride, cdiv for card; see UDiv).
constexpr int32_t kInitChunk = 8192;
constexpr int kInitPerThread = 8;   // entries per thread per pass, sharing each descriptor load

// Unsigned 32-bit division by an invariant divisor d >= 1 as a multiply
// and two shifts (Granlund and Montgomery, "Division by invariant integers
// using multiplication", PLDI 1994, Sec. 4): with l = ceil(log2 d) and
// mul = floor(2^32 (2^l - d) / d) + 1, n / d = (t + ((n - t) >> sh1)) >> sh2
// where t = mulhi(mul, n), sh1 = min(l, 1), sh2 = max(l - 1, 0); exact for
// every n < 2^32.
struct UDiv {
  uint32_t mul;
  uint16_t sh1, sh2;
};
struct InitItem {
  int32_t clique, start;
};
// A clique's CPTs are stored contiguously ([vals_off, vals_off + nvals) of
// the value array, each factor's val_off relative to vals_off), so a CTA can
// stage them in shared memory when they fit kInitSmemBytes.
constexpr int kInitSmemBytes = 32768;
struct InitClique {
  int64_t base_off, vals_off;
  int32_t n, f0, nf, pow2, nvals, pad;
};
struct InitFactor {
  int64_t val_off;
  int32_t t0, nt;
};
struct InitTerm {
  UDiv pdiv, cdiv;
  int32_t shift, card, fstride, pad;
};
template <typename T>
cudaError_t launch_init_cliques(T* base, const InitItem* items, int32_t n_items, const InitClique* cliques,
                                const InitFactor* factors, const InitTerm* terms, const T* vals, int n_sm,
                                cudaStream_t s);
// A permuted table read back in its listed order, as double.
template <typename T>
cudaError_t launch_table_unpermute(const T* table, const CliqueOut& co, double* out_dev, cudaStream_t s);

// The padded plan's tables from the resident ones (FP32): entry e of a
// padded table, read as digits of the padded cardinalities, is the resident
// entry with the same digits, or zero where a digit is an added state.  Run
// after every change of the resident tables.
cudaError_t launch_pad_tables(const float* base, float* pad, const int4* digits, const PadClique* cliques,
                              int32_t n_cliques, int64_t max_pad, cudaStream_t s);

}  // namespace jt

// Internal structures shared by the host planner (jt_plan.cpp), the C ABI
// (jt_capi.cpp) and the kernels (jt_kernels.cu).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/jt.h"

namespace jt {

// ---------------------------------------------------------------------------
// Device-side descriptors (plain structs, copied to device memory once).
//
// Every clique table is stored with its variables permuted: the variables of
// the separator towards the parent come first (most significant digits), in
// ascending variable id, followed by the other variables.  Because of that the
// entries of one parent-separator entry j are the contiguous run
// [j*L, (j+1)*L) of the clique table (L = entries per separator entry), and the
// marginalisation of Eq. 2 towards the parent is a segmented reduction.
//
// Any other table over a subset of the clique's variables (a child separator,
// a single variable for marginals) is indexed by a "key" computed from the
// clique's flat index e with a short list of digit runs ("fields"): a field is
// a maximal run of consecutive clique positions that is also consecutive (and
// in the same order) in the small table's layout:
//     key(e) = sum_f ((e / f.st) % f.len) * f.w
// When every cardinality of the clique is a power of two the same fields are
// evaluated with shifts and masks.
// ---------------------------------------------------------------------------

struct DevField {
  int32_t st;         // clique stride of the run's fastest position
  int32_t len;        // product of the run's cardinalities
  uint32_t st_magic;  // ceil(2^32 / st) (st > 1)
  uint32_t len_magic; // ceil(2^32 / len)
  int32_t w;          // stride of the run's fastest variable in the small table
  int32_t sh;         // log2(st) when the clique is all powers of two
  int32_t lbits;      // log2(len) when the clique is all powers of two
  int32_t pad;
};

struct DevPos {       // one position (digit) of a clique's permuted layout
  int32_t var;
  int32_t card;
  int32_t st;
  uint32_t st_magic;
  uint32_t card_magic;
  int32_t sh;         // log2(st) (power-of-two cliques)
  int32_t cbits;      // log2(card) (power-of-two cliques)
  int32_t pad;
};

struct DevChild {     // a child separator seen from the parent clique
  int32_t child;      // child clique id
  int32_t sep_size;   // entries of the separator table
  int32_t sep_off;    // offset of the separator in per-case message arrays
  int32_t n_field;
  int32_t field_first;
  int32_t w_last;     // key increment per unit of the fastest digit
  int32_t pad0, pad1;
};

struct DevHome {      // a variable whose marginal is read from this clique
  int32_t var;
  int32_t pos;        // its position in the clique's permuted layout
  int32_t card;
  int32_t moff;       // offset of its marginal in per-case marginal arrays
};

struct DevSrc {       // a variable whose marginal is read from this clique's
  int32_t var;        // parent separator once the distribute pass filled it
  int32_t card;
  int32_t st;         // stride of the variable in the separator table
  int32_t moff;
};

struct DevClique {
  int64_t base_off;   // element offset of the (permuted, padded) table
  int32_t n;          // entries
  int32_t k;          // variables
  int32_t L;          // entries per parent-separator entry (n / sep_size)
  uint32_t L_magic;   // ceil(2^32 / L) (L > 1)
  int32_t sep_size;   // parent-separator entries (1 for the root)
  int32_t sep_off;    // offset of that separator in per-case message arrays
  int32_t n_child, child_first;
  int32_t n_home, home_first;
  int32_t n_src, src_first;
  int32_t pos_first;  // k DevPos entries
  int32_t pow2;       // all cardinalities are powers of two
  int32_t card_last;  // cardinality of the fastest position
  int32_t depth;
};

// One CTA's slice of work in a level launch.
struct DevWork {
  int32_t clique;
  int32_t t0, t1;     // entry range [t0, t1), t0 a multiple of the vector width
  int32_t tile;       // index of this slice within the clique (0 writes per-clique scalars)
};

// Kernel arguments for one level launch.
template <typename T>
struct LevelArgs {
  const DevClique* cl;
  const DevPos* pos;
  const DevChild* ch;
  const DevHome* hm;
  const DevSrc* src;
  const DevField* fld;
  const T* base;
  const DevWork* work;
  int32_t case0, n_cases, cb;   // case range and case-block size
  const int16_t* ev;            // [max_cases][n_vars]
  int32_t n_vars;
  T* acc;                       // per case: [up msg_total][down msg_total][marg marg_total]
  int64_t acc_stride;
  int32_t msg_total, marg_total;
  double* ls;                   // [max_cases][n_cliques] log scale of each collect message
  int32_t n_cliques;
  int32_t* status;              // [max_cases]
  T* calib;                     // [max_cases][base_len] or null
  int64_t calib_stride;
  int32_t smem_fac, smem_out;   // per-case smem floats for factors and outputs
};

template <typename T>
struct FinalArgs {
  const int32_t* card_of;       // [n_vars]
  const int32_t* moff;          // [n_vars]
  int32_t n_vars, n_cliques;
  int32_t case0, n_cases;
  const T* acc;
  int64_t acc_stride;
  int32_t msg_total, marg_total;
  int32_t root_sep_off;
  const double* ls;
  int32_t* status;
  double* marg_out;             // [max_cases][marg_total]
  double* logz_out;             // [max_cases]
};

// ---------------------------------------------------------------------------
// Host-side plan.
// ---------------------------------------------------------------------------

struct Plan {
  int32_t n_vars = 0, n_cliques = 0, max_depth = 0;
  std::vector<int32_t> card;
  std::vector<std::vector<int32_t>> vars;   // listed (user) order
  std::vector<std::vector<int32_t>> pvars;  // permuted (device) order
  std::vector<int32_t> parent, depth;
  std::vector<std::vector<int32_t>> children;
  std::vector<std::vector<int32_t>> levels; // cliques per depth
  std::vector<int64_t> n_entries, base_off;
  int64_t base_len = 0;                     // padded element count
  std::vector<std::vector<int32_t>> sep;    // separator vars of edge (c, parent c), ascending
  std::vector<int32_t> sep_size, sep_off;
  int32_t msg_total = 0;
  std::vector<int32_t> home, moff;          // per variable
  std::vector<int32_t> src_edge;            // per variable: separator it is read from, or -1
  int32_t marg_total = 0;
  int64_t entries = 0, work_per_case = 0;

  std::vector<DevClique> dcl;
  std::vector<DevPos> dpos;
  std::vector<DevChild> dch;
  std::vector<DevHome> dhm;
  std::vector<DevSrc> dsrc;
  std::vector<DevField> dfld;
  // per clique: smem floats per case for the collect and distribute passes
  std::vector<int32_t> fac_collect, out_collect_per_seg, fac_dist, out_dist;
};

// Validation + planning from a descriptor.  Returns JT_OK or an error status
// with `err` filled.  Touches no CUDA API.
jt_status build_plan(const jt_tree_desc* d, Plan* p, std::string* err);

// Copy the caller's tables (listed order, any dtype) into the permuted,
// padded device layout (host buffer of base_len elements of T).
template <typename T>
void permute_tables(const Plan& p, const void* pot, jt_dtype pot_dtype, T* out);

uint32_t magic_for(uint32_t d);

}  // namespace jt

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
// Every clique table is stored with its variables permuted:
//   [parent-separator variables, ascending id]   (most significant digits)
//   [variables of child separators, ascending]
//   [private variables]                           (fastest digits)
// A private variable belongs to no separator, so it appears in this clique
// only.  The trailing private variables (product of cardinalities P, the
// "columns") never enter a separator index, a factor or the parent segment:
// viewed as a matrix of rows x P columns, every per-row quantity (factors,
// keys, ratio) is computed once per row, and each entry only costs a
// multiply-add.  Because the parent-separator variables are the slowest
// digits, the rows of one parent-separator entry j form the contiguous run
// [j*LR, (j+1)*LR): marginalisation towards the parent (Eq. 2) is a
// segmented reduction.
//
// Other tables over a subset of the row variables (a child separator) are
// indexed by a key computed from the row index r with digit-run "fields":
// a field is a maximal run of consecutive row positions that is also
// consecutive (in the same order) in the small table's layout:
//     key(r) = sum_f ((r / f.st) % f.len) * f.w
// When every cardinality is a power of two the fields use shifts and masks.
// ---------------------------------------------------------------------------

struct DevField {
  int32_t st;         // row stride of the run's fastest position
  int32_t len;        // product of the run's cardinalities
  uint32_t st_magic;  // ceil(2^32 / st) (st > 1)
  uint32_t len_magic; // ceil(2^32 / len)
  int32_t w;          // stride of the run's fastest variable in the small table
  int32_t sh;         // log2(st) (power-of-two cliques)
  int32_t lbits;      // log2(len) (power-of-two cliques)
  int32_t pad;
};

struct DevPos {       // one position (digit) of a clique's permuted layout
  int32_t var;
  int32_t card;
  int32_t st;         // row positions: row stride; column positions: column stride
  uint32_t st_magic;
  uint32_t card_magic;
  int32_t sh;         // log2(st) (power-of-two cliques)
  int32_t cbits;      // log2(card) (power-of-two cliques)
  int32_t is_col;     // 1 for a column (private suffix) position
};

struct DevChild {     // a child separator seen from the parent clique
  int32_t child;      // child clique id
  int32_t sep_size;   // entries of the separator table
  int32_t sep_off;    // offset of the separator in per-case message arrays
  int32_t n_field;
  int32_t field_first;
  int32_t field_rel;  // field_first relative to the clique's first child field
  int32_t fac_off;    // offset of this table in the clique's per-case factor/output block
  int32_t w_last;     // key step of the clique's fastest digit (0 if that variable is not in the separator)
};

struct DevHome {      // a private variable at a row position: its marginal is
  int32_t pos;        // accumulated per row in this clique's distribute pass
  int32_t card;
  int32_t moff;       // offset of its marginal in per-case marginal arrays
  int32_t out_off;    // offset of its accumulator in the clique's per-case output block
};

struct DevSrc {       // a variable whose marginal is binned from a small table:
  int32_t var;        // a separator (DevClique.src_*) or the column joint
  int32_t card;       // (DevClique.jh_*)
  int32_t st;         // stride of the variable in that table
  int32_t moff;
};

struct DevClique {
  int64_t base_off;   // element offset of the (permuted, padded) table
  int32_t n;          // entries
  int32_t k;          // variables
  int32_t kr;         // row positions 0..kr-1; column positions kr..k-1
  int32_t P;          // columns (product of the column cardinalities), >= 1
  uint32_t P_magic;
  int32_t logP;
  int32_t LR;         // rows per parent-separator entry
  uint32_t LR_magic;
  int32_t logLR;
  int32_t sep_size;   // parent-separator entries (1 for the root)
  int32_t sep_off;    // offset of that separator in per-case message arrays
  int32_t n_child, child_first;
  int32_t n_home, home_first;   // private variables at row positions
  int32_t n_jh, jh_first;       // private variables in the columns (DevSrc, stride in the joint)
  int32_t joint_off;            // offset of the column joint in per-case arrays (-1: none)
  int32_t n_src, src_first;     // variables read from the parent separator
  int32_t pos_first;            // k DevPos entries
  int32_t pow2;                 // all cardinalities are powers of two
  int32_t depth;
  int32_t field_first, n_field; // fields of all child separators (contiguous)
  int32_t card_last;            // cardinality of the fastest position
  // offsets (entries) of this clique's tables inside the per-case shared-memory
  // table region of a propagation, or -1 when the table stays in global memory
  int32_t sm_fac;               // child factors (collect messages of the children)
  int32_t sm_rho;               // parent ratio
  int32_t sm_out;               // child-separator and row-home accumulators
  int32_t sm_jnt;               // column joint
  int32_t sm_out_len;           // entries of the accumulators (child separators + row homes)
};

// One work item of a propagation: a slice of one clique's table for one
// block of evidence cases, in one pass.
struct DevWork {
  int64_t base_off;   // element offset of the clique's table (copied from DevClique)
  int32_t clique;
  int32_t t0, t1;     // entry range [t0, t1), t0 a multiple of the chunk
  int32_t ntiles;     // slices of this clique (per case block and pass)
  int32_t cbk;        // case block
  int32_t collect;    // 1: collect pass, 0: distribute pass
};

// Kernel arguments for one level launch.
//
// Per-case array (stride acc_stride elements):
//   [up: msg_total]    collect messages; raw sums, normalised to mean one in
//                      place by the last CTA of the sending clique
//   [down: msg_total]  distribute messages (raw sums)
//   [rho: msg_total]   parent ratios new/old (0/0 := 0), written by the last
//                      CTA of the parent clique
//   [marg: marg_total] raw marginal sums
//   [joint: joint_total] column joints of cliques with private variables
template <typename T>
struct LevelArgs {
  const DevClique* cl;
  const DevPos* pos;
  const DevChild* ch;
  const DevHome* hm;
  const DevSrc* src;
  const DevSrc* jh;
  const DevField* fld;
  const T* base;
  const DevWork* work;
  int32_t case0, n_cases, cb;   // case range and case-block size
  const int16_t* ev;            // [max_cases][n_vars]
  int32_t n_vars;
  T* acc;
  int64_t acc_stride;
  int32_t msg_total, marg_total, joint_total;
  double* ls;                   // [max_cases][n_cliques] log scale of each collect message
  int32_t n_cliques;
  int32_t* status;              // [max_cases]
  int32_t* cnt;                 // [2][n_cliques][max_cases] tile tickets (self-resetting)
  int32_t* done;                // [2][n_cliques][max_cases] messages final (zeroed per propagation)
  int32_t* queue;               // next work item (zeroed per propagation)
  int32_t n_items;
  const int32_t* parent_of;     // [n_cliques]
  int32_t* err;                 // device error word (set on a timed-out wait)
  int32_t max_cases;
  T* calib;                     // [max_cases][base_len] or null
  int64_t calib_stride;
};

// Where the finalisation reads a variable's marginal from (per-case offsets).
struct VarSrc {
  int64_t off;        // kind 1: start of the table; kind 0: start of the raw marginal
  int32_t kind;       // 1: bin a separator table or a column joint; 0: raw sums per state
  int32_t card;
  int32_t st;         // stride of the variable in the table (kind 1)
  int32_t size;       // table entries (kind 1)
  int32_t moff;       // offset of the marginal in the output
  int32_t pad;
};

template <typename T>
struct FinalArgs {
  const VarSrc* vs;             // [n_vars]
  int32_t n_vars, n_cliques;
  int32_t case0, n_cases;
  const T* acc;
  int64_t acc_stride;
  int32_t msg_total, marg_total;
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
  std::vector<DevSrc> dsrc, djh;
  std::vector<DevField> dfld;
  int32_t joint_total = 0;
  std::vector<VarSrc> vsrc;                 // per variable
  // per clique: per-case shared-memory entries of the child factors and of
  // the distribute outputs (child separators + row-home marginals)
  std::vector<int32_t> fac_collect, out_dist;
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

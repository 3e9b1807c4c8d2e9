// Internal structures shared by the host planner (jt_plan.cpp), the C ABI
// (jt_capi.cpp) and the kernels (jt_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/jt.h"

namespace jt {

// ---------------------------------------------------------------------------
// Layout (planned once per tree, see build_plan).
//
// Every clique table is stored with its variables permuted ("positions",
// position 0 most significant):
//   [parent-separator variables, in the order they have in the parent]
//   [variables shared with child separators, most-shared first]
//   [private variables (in no separator)]                   (fastest digits)
// and every separator table is laid out in the order its variables have in
// the parent clique (first most significant).  So for any small table over a
// subset V of a clique's variables (a separator, or the joint of the private
// variables) the table key of an entry is the clique index with the digits
// outside V dropped:
//     key(x) = sum_f ((x / f.st) % f.len) * f.w
// over "fields" = maximal runs of consecutive positions inside V.  The key is
// additive over disjoint digit sets, so for a block of the table that fixes
// every digit above some position, key(block_start + o) = key(block_start)
// + key(o): the block touches the contiguous key window
// [key(block_start), key(block_start) + K), K = product of the cardinalities
// of V's positions inside the block.  When every cardinality is a power of
// two the digits are bit fields and blocks may cut a digit.
// ---------------------------------------------------------------------------

// Port kinds: the small tables one clique touches in one pass.
constexpr int32_t kPortMu = 0;     // in : collect message of a child, normalised to mean one
constexpr int32_t kPortRho = 1;    // in : ratio new/old of the clique's own parent separator (0/0 := 0)
constexpr int32_t kPortU = 2;      // out: collect message to the parent (raw sums)
constexpr int32_t kPortDelta = 3;  // out: distribute message to a child (raw sums)
constexpr int32_t kPortJoint = 4;  // out: joint of the private variables (raw sums)

// Optional per-item trace (global timer, ns): SM, consumers start, item
// prepared, streaming starts, streamed, consumers done, time consumer thread 0
// waited for chunks, producer took the item, producer issued its last chunk,
// block published.
constexpr int kTraceSlots = 12;

constexpr int kStatusZero = 1;      // P(e) = 0
constexpr int kStatusBadState = 2;  // an evidence state >= card

struct DevField {
  int32_t st;         // entry stride of the run's fastest position
  int32_t len;        // product of the run's cardinalities
  uint32_t st_magic;  // ceil(2^32 / st)
  uint32_t len_magic; // ceil(2^32 / len)
  int32_t w;          // stride of the run's fastest variable in the small table
  int32_t sh;         // power-of-two cliques: log2(st)
  int32_t lb;         // power-of-two cliques: log2(len)
  int32_t pad;
};

struct DevPos {       // one digit (position) of a clique's permuted layout
  int32_t var;
  int32_t card;
  int32_t st;         // entry stride
  uint32_t st_magic;
  uint32_t card_magic;
  int32_t sh;         // power-of-two cliques: log2(st)
  int32_t cb;         // power-of-two cliques: log2(card)
  int32_t card_ev;    // evidence states must lie below this: the variable's
                      // cardinality before any padding to a power of two
};

constexpr int32_t kVmodeStore = 4;
constexpr int64_t kFineJointEntries = 64;  // largest joint of the case-block layout
struct DevPort {
  int32_t kind;       // kPort*
  int32_t tab;        // offset of the table in the per-case message array
  int32_t size;       // entries of the table
  int32_t K;          // entries of the window a block touches
  int32_t win;        // offset of the window in the per-case window region
  int32_t other;      // kPortMu: the child clique; kPortRho: this clique
  int32_t other2;     // kPortRho: the parent clique
  int32_t nf;         // fields
  int32_t f0;         // first field (index relative to the stage's first field)
  uint32_t lane_free; // fast path: lane bits the key does not depend on
  int32_t vmode;      // fast path: a vector's entries have keys key0 + dvec[j]: 0 = all dvec 0,
                      // 1 = dvec[j] = j, 2 = other; | kVmodeStore: an output whose window
                      // has one entry per block entry (no two entries share a key)
  int32_t dvec[4];    // fast path: key offsets of the entries of a vector
  int32_t iter_dep;   // fast path: bit 0: the key depends on the iteration bits (entry bits above
                      // the thread's vector index); bit 1: on the chunk bits (above one chunk);
                      // bit 2: on the iteration bits inside one chunk
};

// One clique in one pass.
struct DevStage {
  int64_t base_off;   // element offset of the permuted table
  int32_t clique, pass;   // pass 0 = collect (Algorithm 2), 1 = distribute (Algorithm 3)
  int32_t n;          // entries
  int32_t B;          // entries of one block (one work item)
  int32_t n_blocks;
  int32_t k;          // positions
  int32_t kin;        // generic path: positions [k - kin, k) lie inside a block
  int32_t bits;       // fast path: log2(B); -1 selects the generic path
  int32_t pos0;       // first DevPos
  int32_t np, nin;    // ports, of which [0, nin) are inputs
  int32_t port0;      // first DevPort
  int32_t nf, field0; // fields of all ports
  int32_t win_len;    // per-case window entries
  int32_t ndep, dep0; // dependencies: pairs (stage, blocks) in the dependency list
  int32_t sum_slot;   // index of this stage's total in the per-case sums (pass * n_cliques + clique)
  // fast path: the ports with windows and their key tables, precomputed and
  // carried in the stage's descriptor blob (byte offsets from its start):
  // LivePort[n_live] at live_off, then int32 kiter[n_live][kMaxIter] (entries
  // past the block's n_iter repeat its last one), then uint16
  // kt[n_live][consumers]
  int32_t n_live, n_in_live;  // ports with windows, of which [0, n_in_live) are inputs
  int32_t n_iter;             // consumer iterations of one block
  int32_t live_off;
  // positions (bit i = position i) whose variable is in some input port of
  // the stage: evidence on such a variable inside a block already zeroes
  // that input's window entries (the message it carries was computed with
  // the evidence), so the case-lane schedule masks only the other positions
  uint32_t covered;
  // padded plans: up to three digits lying above the 32-entry tile whose
  // added states make a whole tile of zero entries (a tile with such a digit
  // at an added state contributes nothing), packed as
  // shift | bits << 5 | original cardinality << 10; 0 = none
  uint32_t holes[3];
};

// A port with a window, as the fast path reads it.  An entry at block offset
// o = m * (consumers * VEC) + tid * VEC + j has the key
// kt[port][tid] + kiter[port][m] + dvec[j] (kt includes the window start).
struct LivePort {
  int32_t mode;       // bits 0-1 vmode, bit 2 key depends on the iteration, bits 3-7 lane_free,
                      // bit 8 key depends on the chunk, bit 9 the window is the block itself,
                      // bit 10 key depends on the iteration inside a chunk (without it, a
                      // thread's vectors of one chunk share their keys)
  int32_t port;
  int32_t win;        // start of the port's window (in every case's window row)
  int32_t pad;
  int32_t dvec[4];
};
static_assert(sizeof(LivePort) == 32 && offsetof(LivePort, win) == 8 && offsetof(LivePort, dvec) == 16,
              "live-port table layout");
constexpr int32_t kModeIter = 4;
constexpr int32_t kModeChunk = 256;
constexpr int32_t kModeStore = 512;
constexpr int32_t kModeInChunk = 1024;

// Byte offsets of the key tables inside a stage blob.
__host__ __device__ inline int32_t kiter_off(const DevStage& S) { return S.live_off + S.n_live * 32; }
constexpr int kMaxIter = 64;                    // consumer iterations of one fast-path block
__host__ __device__ inline int32_t kt_off(const DevStage& S) { return kiter_off(S) + S.n_live * kMaxIter * 4; }

static_assert(sizeof(DevField) % 16 == 0 && sizeof(DevPos) % 16 == 0, "descriptor blobs are 16-byte granular");
static_assert(sizeof(DevPort) % 16 == 0 && sizeof(DevStage) % 16 == 0, "descriptor blobs are 16-byte granular");

// One work item: one block of one stage for one block of evidence cases.
struct DevItem {
  int64_t off;        // element offset of the block's first entry in the table array
  int32_t n;          // entries of the block
  int32_t stage;
  int32_t block;
  int32_t cbk;        // case block
  int32_t blob;       // the stage's descriptor blob: offset in 16-byte units
  int32_t blob_bytes; //   and size (DevStage, DevPort[np], DevField[nf], DevPos[k])
};

// Where the finalisation reads a variable's marginal: a separator's
// distribute message or a clique's private joint (per-case offsets).
struct VarSrc {
  int32_t off;        // start of the table in the per-case message array
  int32_t size;       // table entries
  int32_t st;         // stride of the variable in the table
  int32_t card;
  int32_t moff;       // offset of the marginal in the output row
  int32_t card_out;   // states written to the marginal row (the cardinality
                      // before padding; padded states are zero)
  int32_t pad[2];
};

// Arguments of the persistent propagation kernel.
template <typename T>
struct PropArgs {
  const T* base;                // permuted clique tables
  const DevStage* stages;
  const DevPort* ports;
  const DevField* fields;
  const DevPos* pos;
  const int32_t* deps;          // pairs (stage, blocks)
  const uint4* blobs;           // per-stage descriptor blobs
  const DevItem* items;
  int32_t n_items;
  int32_t case0, n_cases;       // case range of this propagation
  int32_t n_cb;                 // case blocks
  const int16_t* ev;            // [max_cases][n_vars], -1 = unobserved
  int32_t n_vars;
  T* msg;                       // [max_cases][msg_stride]: u | delta | joint
  int64_t msg_stride;
  int32_t delta_off;            // start of the distribute messages in a message row
  double* sums;                 // [max_cases][2 * n_cliques]: collect totals (sigma), distribute totals (Delta)
  int32_t n_cliques;
  int32_t* status;              // [max_cases]
  int32_t* done;                // [n_stages][n_cb] finished blocks
  int32_t* queue;               // next work item
  int32_t* err;                 // set when a bounded wait gives up
  uint64_t wait_ns;             // limit of every bounded device-side wait (ns)
  T* calib;                     // [max_cases][calib_stride] calibrated tables, or null
  int64_t calib_stride;
  uint64_t* trace;              // [n_items][kTraceSlots] item timeline, or null
  unsigned long long* span;     // [2]: first CTA start, last CTA end (global timer, ns), or null
  // shared-memory plan
  int32_t ring;                 // bulk-copy stages
  int32_t chunk;                // entries per stage
  int32_t max_k, max_ports, max_fields, win_max;
  int32_t blob_max;             // bytes of the largest stage blob
};

template <typename T>
struct FinalArgs {
  const VarSrc* vs;             // [n_vars]
  int32_t n_vars, n_cliques;
  int32_t case0, n_cases;
  const T* msg;
  int64_t msg_stride;
  const double* sums;
  const int32_t* sep_size;      // [n_cliques]
  int32_t* status;
  int32_t marg_total;
  double* marg_out;             // [max_cases][marg_total]
  double* logz_out;             // [max_cases]
  int32_t lanes;                // cases interleaved in a message slab (1: one row per case)
  // case lanes: the variables, those whose source table holds at most
  // kFinWarpEntries entries first (a warp each), then the others (a CTA each)
  const int32_t* var_order;
  int32_t n_small;
};
constexpr int32_t kFinWarpEntries = 256;

// The finalisation order of a marginal-source layout (small sources first).
inline std::vector<int32_t> fin_order(const std::vector<VarSrc>& vs, int32_t* n_small) {
  std::vector<int32_t> order;
  for (int v = 0; v < (int)vs.size(); ++v)
    if (vs[v].size <= kFinWarpEntries) order.push_back(v);
  *n_small = (int32_t)order.size();
  for (int v = 0; v < (int)vs.size(); ++v)
    if (vs[v].size > kFinWarpEntries) order.push_back(v);
  return order;
}

// ---------------------------------------------------------------------------
// Host-side plan of a tree (independent of the case-block size).
// ---------------------------------------------------------------------------
struct Plan {
  int32_t n_vars = 0, n_cliques = 0, max_depth = 0;
  std::vector<int32_t> card;
  // A padded plan (build_padded_plan): every cardinality raised to a power of
  // two, the added states impossible (their potential entries zero), and
  // card_ev the cardinalities of the tree it pads; empty otherwise.
  std::vector<int32_t> card_ev;
  std::vector<std::vector<int32_t>> vars;   // listed (user) order
  std::vector<std::vector<int32_t>> pvars;  // permuted (device) order
  std::vector<int32_t> parent, depth;
  std::vector<std::vector<int32_t>> children;
  std::vector<std::vector<int32_t>> levels; // cliques per depth
  std::vector<int64_t> n_entries, base_off;
  std::vector<uint8_t> pow2;                // every cardinality of the clique is a power of two
  int64_t base_len = 0;                     // padded element count of all tables
  std::vector<std::vector<int32_t>> sep;    // separator of (c, parent c), in the parent's permuted order
  std::vector<int32_t> sep_size, sep_off;   // root: a 1-entry slot
  int32_t msg_total = 0;                    // entries of all separator tables
  std::vector<int32_t> n_private;
  // Private-variable joints, in three layouts, each a list of joints per
  // clique over consecutive private positions.  Layout 0: one joint over all
  // of a clique's private variables (one-case schedules accumulate it in
  // registers).  Layout 1: joints of at most kFineJointEntries entries
  // (case-block schedules keep a window per case and joint in shared memory,
  // so the windows must stay small for blocks to stay large).  Layout 2: one
  // joint per private variable -- its marginal is all the finalisation needs
  // -- for case-lane schedules, whose reductions into a window cost per
  // distinct key of a tile.
  struct JointGroup {
    int32_t off, size;                      // offset in the joint region, entries
    int32_t pos0, npos;                     // permuted positions [pos0, pos0 + npos)
  };
  std::vector<std::vector<JointGroup>> joints[3];
  int32_t joint_total = 0;                  // both layouts
  std::vector<int32_t> moff;                // per variable: offset of its marginal
  int32_t marg_total = 0;
  std::vector<VarSrc> vsrc[3];              // per layout, per variable (offsets in a message row)
  int64_t entries = 0, work_per_case = 0;
  int64_t msg_stride = 0;                   // u | delta | joint, padded
};

// Validation + layout.  Returns JT_OK or an error status with `err` filled.
// Touches no CUDA API.
jt_status build_plan(const jt_tree_desc* d, Plan* p, std::string* err);

// The tree of `p` with every cardinality raised to the next power of two.
// The added states get zero potential in every clique that holds the
// variable, so the padded tree has the same joint distribution on the
// original states, the same normalising constant and the same marginals
// (Eq. 1: every product with a zero entry vanishes).  The permuted variable
// order of every clique is the one of `p` (it does not depend on
// cardinalities); marginal offsets and evidence limits are those of `p`, so
// a propagation over the padded plan writes the same output rows.
// JT_ERR_UNSUPPORTED if the padded tables would exceed the layout's limits.
jt_status build_padded_plan(const Plan& p, Plan* q, std::string* err);

// Map from a plan's permuted tables to its padded plan's: per clique, per
// permuted position, the padded shift and width and the original cardinality
// and stride (int4 {sh, bits, card, stride}), and per clique where its digits
// and both of its tables start.
struct PadClique {
  int64_t off, off_pad, n_pad;  // table offsets (original, padded), padded entries
  int32_t d0, k;                // digits [d0, d0 + k)
};
struct PadMap {
  std::vector<int4> digits;
  std::vector<PadClique> cliques;
};
PadMap build_pad_map(const Plan& p, const Plan& q);

// Copy the caller's tables (listed order, any dtype) into the permuted,
// padded device layout (host buffer of base_len elements of T).
template <typename T>
void permute_tables(const Plan& p, const void* pot, jt_dtype pot_dtype, T* out);

// Clique-size classes of the block-size tuning: tables of fewer than 2^14
// entries, fewer than 2^18, and larger.
constexpr int kBlockClasses = 3;
inline int block_class(int64_t entries) { return entries < (1 << 14) ? 0 : entries < (1 << 18) ? 1 : 2; }

// Schedule of one propagation shape (case-block size): stages, ports,
// fields, dependencies and the ordered work items.
struct Schedule {
  int32_t cb = 1, n_cb = 1;
  int8_t block_shift[kBlockClasses] = {0, 0, 0};  // the block-target shifts it was planned with
  std::vector<DevStage> stages;             // [2 * n_cliques]; the root's collect stage is empty
  std::vector<DevPort> ports;
  std::vector<DevField> fields;
  std::vector<DevPos> pos;
  std::vector<int32_t> deps;
  std::vector<uint4> blobs;                 // per stage: DevStage, DevPort[np], DevField[nf], DevPos[k],
                                            // and on the fast path the live ports and key tables
  std::vector<DevItem> items;
  int32_t ring = 0, chunk = 0;
  int32_t max_k = 1, max_ports = 1, max_fields = 1, win_max = 1;
  int32_t blob_max = 16;                    // bytes of the largest stage blob
  int64_t streamed_entries = 0;             // entries streamed per case block (all stages)
  // whole-tree schedules (cb == kWholeTree): one CTA propagates one case at a
  // time, level by level (see SmallPlan)
  struct SmallPlan {
    std::vector<uint4> blobs;               // each level's stage descriptors (DevStage, ports, fields,
                                            // positions), level after level
    std::vector<int32_t> lv_blob_off;       // [levels + 1] first 16-byte unit of each level's descriptors
    int32_t lv_blob_max = 0;                // 16-byte units of the largest level
    std::vector<int32_t> stage_blob;        // [2 n_cliques] a stage's descriptors within its level's
                                            // (16-byte units), -1: empty
    std::vector<int2> segs;                 // (stage, first entry) of every segment, level by level
    std::vector<int32_t> seg_lv;            // [levels + 1] first segment of each level
    std::vector<int32_t> lv_stage;          // the stages of each level
    std::vector<int32_t> lv_stage_off;      // [levels + 1]
    int32_t levels = 0;
    int32_t smem = 0;                       // dynamic shared memory of one CTA
    bool base_in_smem = false;              // the clique tables fit beside the rest: staged once per CTA
    bool desc_resident = false;             // every level's descriptors fit (lv_blob_max is then all
                                            // of them): staged once per CTA
    // every index array above and the separator sizes, packed (int32) for
    // one copy into shared memory: lv_blob_off | seg_lv | lv_stage_off |
    // stage_blob | lv_stage | sep_size | segs (as pairs), each part starting
    // on an even element; offsets of the parts
    std::vector<int32_t> idx;
    int32_t o_seg_lv = 0, o_lv_stage_off = 0, o_stage_blob = 0, o_lv_stage = 0, o_sep_size = 0, o_segs = 0;
    bool idx_in_smem = false;               // the packed indices fit too: staged once per CTA
  } small;
};

// Cases per work item of a whole-tree schedule (reported as 0): every case
// of the range is one work item, propagated by one CTA from its shared memory.
constexpr int kWholeTree = 0;
constexpr int kSmallSeg = 32;               // entries of one segment (a warp's share of a clique)

// Plan the schedule for `n_cases` cases in blocks of `cb` on a device with
// `n_sm` SMs and `smem_bytes` of dynamic shared memory per CTA.  A stage's
// block size is the largest power of two (or digit product) within a target
// that spreads its level over the SMs and within the shared-memory budget of
// its windows; `block_shift` (per clique-size class, or null) scales that
// target by 2^shift before the hard limits apply.
jt_status build_schedule(const Plan& p, int elem, int cb, int n_cases, int n_sm, int smem_bytes,
                         Schedule* s, std::string* err, const int8_t* block_shift = nullptr);

// Plan a whole-tree schedule (one CTA per case): the one-case stage
// descriptors plus the level-ordered segment list.  JT_ERR_UNSUPPORTED when
// the tree's per-case state does not fit one CTA's shared memory or the tree
// is too large for one CTA to propagate efficiently.
jt_status build_small_schedule(const Plan& p, int elem, int n_cases, int n_sm, int smem_bytes, Schedule* s,
                               std::string* err);

// Arguments of the whole-tree propagation kernel.
template <typename T>
struct SmallArgs {
  const T* base;                // permuted clique tables
  const uint4* blobs;           // level-ordered stage descriptors
  int32_t lv_blob_max;          // 16-byte units of the largest level (its shared-memory staging)
  // packed indices (Schedule::SmallPlan::idx): lv_blob_off [levels + 1],
  // seg_lv [levels + 1], lv_stage_off [levels + 1], stage_blob [2 n_cliques]
  // (within the level's descriptors), lv_stage, sep_size [n_cliques], segs
  const int32_t* idx;
  int32_t idx_len;              // elements (a multiple of 4)
  int32_t o_seg_lv, o_lv_stage_off, o_stage_blob, o_lv_stage, o_sep_size, o_segs;
  int32_t idx_in_smem;
  int32_t levels;
  const int16_t* ev;            // [max_cases][n_vars], -1 = unobserved
  int32_t n_vars;
  T* msg;                       // [max_cases][msg_stride]: u | delta | joint
  int64_t msg_stride;
  int32_t msg_total;            // entries of the collect (and of the distribute) messages
  double* sums;                 // [max_cases][2 n_cliques]
  int32_t n_cliques;
  int32_t* status;
  int32_t case0, n_cases;
  unsigned long long* span;     // [2] kernel span (global timer), or null
  int32_t base_in_smem;         // copy the clique tables into shared memory once per CTA
  int64_t base_len;             // elements of the clique tables (a multiple of 32)
  int32_t desc_resident;        // every level's descriptors staged once per CTA
  uint64_t* trace;              // [2 + 4 levels] phase times of CTA 0's first case, or null
};

// Dynamic shared memory of the propagation kernel for a schedule.
int32_t prop_smem_bytes(const Schedule& s, int elem);

uint32_t magic_for(uint32_t d);

}  // namespace jt

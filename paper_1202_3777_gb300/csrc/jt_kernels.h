// Launch interface of the propagation kernels (used by the planner and the
// C ABI layer).
#pragma once

#include <cuda_runtime.h>

#include "jt_internal.h"

namespace jt {

// Shape of a propagation CTA for a case-block size: consumer threads (plus
// one producer warp) and resident CTAs per SM.
__host__ __device__ constexpr int consumers_for(int cb) { return cb > 0 ? 512 : 512; }
__host__ __device__ constexpr int ctas_per_sm_for(int cb) { return cb > 0 ? 1 : 1; }
// Bytes per bulk-copy stage: four vectors per consumer thread for one case
// (processed together, so their latencies overlap), one vector for a block
// of cases (eight cases already overlap; their windows need the room).
__host__ __device__ constexpr int chunk_bytes_for(int cb) { return cb > 1 ? 8192 : 32768; }
// Case-lane schedules: a work item carries kCaseLanes evidence cases, one per
// lane of every consumer warp.  All lanes of a warp walk the same entries of
// the streamed block, so the entry walk, the keys and the shared loads of the
// table are common to the cases, and each lane reduces into its own case's
// column of case-minor windows ([key][case]) and message slabs, with no
// cross-lane reduction.
constexpr int kCaseLanes = 32;
constexpr int kClPortBytes = 448;               // bytes of one port's key tables (CLPort, below)
constexpr int kSig = 2;                         // finished items queued for the signalling lane
constexpr int kControlThreads = 96;             // producer, signalling and preparation warps
constexpr int kMaxFastPorts = 16;               // ports of a stage on the power-of-two fast path
constexpr int kClMaxPorts = 32;                 // ports of a stage on the case-lane path (tables in the blob)

// Bytes of a stage's descriptors (DevStage, ports, fields, positions).
__host__ __device__ inline int32_t desc_bytes(int k, int np, int nf) {
  return (int32_t)sizeof(DevStage) + np * (int32_t)sizeof(DevPort) + nf * (int32_t)sizeof(DevField) +
         k * (int32_t)sizeof(DevPos);
}
// Bytes of a fast-path stage's live ports and key tables.
// (one-case and case-lane schedules carry them in the blob; case-block
// schedules compute them per item into shared memory, which leaves their hot
// loop's registers as they are)
__host__ __device__ inline int32_t table_bytes(int cb, int n_live) {
  if (cb == kCaseLanes) return n_live * kClPortBytes;
  return cb == 1 ? n_live * (32 + kMaxIter * 4 + consumers_for(cb) * 2) : 0;
}

// Dynamic shared memory of a propagation CTA, carved identically by the
// planner (host) and the kernel (device).  Everything an item needs besides
// the streamed table (descriptor blob with its key tables, evidence lists,
// block factors, windows) is double-buffered: the control warps prepare item
// i+1 and flush item i-1 while the consumers stream item i.
struct SmemLayout {
  int32_t bar, info, sig, blob, blob_bytes, obs, nobs, bf, pval, red, misc, kiter, live, kt, win, ring, bytes;

  __host__ __device__ static int32_t a16(int32_t x) { return (x + 15) & ~15; }

  __host__ __device__ SmemLayout(int cb, int ring_n, int chunk, int max_k, int max_ports, int blob_max,
                                 int win_max, int elem) {
    int32_t o = 0;
    bar = o;  o += (2 * ring_n + 8 + 2 * kSig) * 8;   // ring full/empty; per buffer: item, blob, prepared,
                                                      // flushed; signal slots full/empty
    info = a16(o);   o = info + 2 * 64;                // per buffer: the item and its preparation status
    sig = a16(o);    o = sig + kSig * 16;              // finished items for the signalling lane
    blob_bytes = a16(blob_max);
    blob = (o + 127) & ~127; o = blob + 2 * blob_bytes;
    obs = a16(o);    o = obs + 2 * cb * max_k * 16;    // in-block observations per case
    nobs = a16(o);   o = nobs + 2 * cb * 4;
    bf = a16(o);     o = bf + 2 * cb * 8;              // block factor per case
    pval = a16(o);   o = pval + 2 * cb * max_ports * 8;  // per (case, input port) factor
    red = a16(o);    o = red + cb * (consumers_for(cb) / 32) * 8;  // block-total partials
    misc = a16(o);   o = misc + 16 * 4;
    kiter = live = kt = 0;
    if (cb > 1) {  // key tables computed per item (case blocks)
      kiter = a16(o);  o = kiter + kMaxFastPorts * kMaxIter * 4;
      live = a16(o);   o = live + kMaxFastPorts * 32;
      kt = a16(o);     o = kt + kMaxFastPorts * consumers_for(cb) * 4;
    }
    win = (o + 127) & ~127;  o = win + 2 * cb * win_max * elem;
    ring = (o + 127) & ~127; o = ring + ring_n * chunk * elem;
    bytes = o;
  }
};

// Key tables of one port of a case-lane stage, built by the planner and
// carried in the stage's descriptor blob (CLPort[n_live] at live_off).  A
// chunk ci of a block is 64 tiles of 32 entries; consumer warp w streams the
// tiles at positions p = w + 16 t (t < kClTiles), interleaved so that a block
// shorter than a chunk still spreads over the warps.  An entry's block offset
// is o = ci * chunk + 32 p + 4 v + j and (power-of-two digits are bit fields)
// its key is the sum of the keys of those parts.
// Every table holds byte offsets into the case-minor windows (key * 128), the
// chunk table also the port's window start, so a lane's address is the item
// buffer's window base plus a sum of table entries plus lane * 4.
constexpr int kClSlice = 128;                   // entries a warp streams from one chunk
constexpr int kClTiles = kClSlice / 32;         // tiles of 32 entries per slice
constexpr int kClMaxChunks = 32;                // chunks of one block (blocks <= 2^16 entries)
constexpr int kClRow = 32 * 4;                  // bytes of one window row (one key, every case)
struct CLPort {
  int32_t cls;                   // kClInput | kClTile, kClVector or kClEntry
  int32_t dep;                   // bit b (b < 5): the key depends on bit b of a tile entry's offset
  int32_t pad[2];
  int32_t dvec[4];               // key(j) * row, j < 4 (entries of a vector)
  int32_t kvec[8];               // key(4 v) * row, v < 8 (vectors of a tile)
  int32_t kslot[16 * kClTiles];  // key(32 p) * row for tile position p of a chunk
  int32_t kchunk[kClMaxChunks];  // port window start + key(ci * chunk) * row (bytes from the buffer's windows)
};
constexpr int32_t kClInput = 1;
constexpr int32_t kClTile = 0;      // key constant over a tile of 32 entries
constexpr int32_t kClVector = 2;    // key constant over each vector of 4 entries
constexpr int32_t kClEntry = 4;     // key changes within a vector
constexpr int32_t kClIdent = 8;     // with kClEntry: the tile's keys are key + e, e < 32 (consecutive rows)
// bits 4-5: register slot + 1 of an output whose key depends only on entry
// bits 0-1 (the same four rows for every tile of a block): its four sums
// accumulate in registers over the block and reduce once per item.  One
// slot: more accumulators were measured slower (they push the hot loop into
// spills).
constexpr int32_t kClRegShift = 4;
constexpr int kClRegSlots = 1;
static_assert(sizeof(CLPort) == kClPortBytes && sizeof(CLPort) % 16 == 0, "case-lane port table");

// Dynamic shared memory of a case-lane propagation CTA (host and device
// carve it alike): barriers, item slots, descriptor blobs (with the port
// tables), then per buffer the evidence masks (V, M per case) and the block
// factor per case (which carries the block totals to the signalling lane
// once the block has streamed), the warps' partial totals, the case-minor
// windows per buffer, and the bulk-copy ring.
struct SmemLayoutCL {
  int32_t bar, info, sig, blob, blob_bytes, ev, bf, misc, red, win, ring, bytes;

  __host__ __device__ static int32_t a16(int32_t x) { return (x + 15) & ~15; }

  __host__ __device__ SmemLayoutCL(int ring_n, int chunk, int blob_max, int win_max) {
    int32_t o = 0;
    bar = o;  o += (2 * ring_n + 8 + 2 * kSig) * 8;
    info = a16(o);   o = info + 2 * 64;
    sig = a16(o);    o = sig + kSig * 16;
    blob_bytes = a16(blob_max);
    blob = (o + 127) & ~127; o = blob + 2 * blob_bytes;
    ev = a16(o);     o = ev + 2 * kCaseLanes * 16;             // per buffer, per case: V, M, -, -
    bf = a16(o);     o = bf + 2 * kCaseLanes * 8;              // per buffer, per case: block factor
    misc = a16(o);   o = misc + 16 * 4;
    red = a16(o);    o = red + kCaseLanes * 16 * 8;            // per case, per warp: partial totals
    win = (o + 127) & ~127;  o = win + 2 * win_max * kClRow;
    ring = (o + 127) & ~127; o = ring + ring_n * chunk * 4;
    bytes = o;
  }
};

// Enqueue one persistent propagation launch of `grid` CTAs (collect and
// distribute of every clique for the case range of `a`).
template <typename T>
cudaError_t launch_propagate(const PropArgs<T>& a, int cb, int grid, int smem, cudaStream_t s);

// Enqueue the finalisation (log Z and normalised marginals) for a case range.
template <typename T>
cudaError_t launch_finalize(const FinalArgs<T>& a, cudaStream_t s);

// Whole-tree schedules: one CTA per case (at a time), the case's messages in
// shared memory; the dynamic shared memory one CTA needs.
int32_t small_smem_bytes(int64_t msg_stride, int32_t msg_total, int32_t n_cliques, int32_t n_vars, int elem,
                         int32_t lv_blob_max);
template <typename T>
cudaError_t launch_small(const SmallArgs<T>& a, int grid, int smem, cudaStream_t s);

// Case-lane schedules (FP32): the persistent propagation over message slabs
// of kCaseLanes interleaved cases, and its finalisation.
cudaError_t launch_propagate_cl(const PropArgs<float>& a, int grid, int smem, bool holes, cudaStream_t s);
cudaError_t launch_finalize_cl(const FinalArgs<float>& a, cudaStream_t s);

// Normalised calibrated clique in the caller's listed order.
struct CliqueOut {
  int32_t n, k;
  int32_t lcard[32];             // listed cardinalities
  int32_t pst[32];               // permuted stride of each listed position
};
// Calibrated-clique read-out: out_dev = the table in listed order, normalised
// to sum one; sum_dev holds ceil(n / kNoAllocPerBlock) partial sums.
template <typename T>
cudaError_t launch_get_clique(const T* calib_clique, const CliqueOut& co, double* out_dev,
                              double* sum_dev, cudaStream_t s);

// Allocation-free calibrated-clique read-out (jt_get_clique_noalloc): the
// normalising sum is reduced through a file-scope device array of
// kNoAllocMaxBlocks partial sums, one per kNoAllocPerBlock table entries, so
// tables of at most kNoAllocMaxEntries entries are accepted.
constexpr int kNoAllocMaxBlocks = 1024;
constexpr int kNoAllocPerBlock = 4096;
constexpr int64_t kNoAllocMaxEntries = (int64_t)kNoAllocMaxBlocks * kNoAllocPerBlock;
constexpr int kNoAllocMaxDevices = 64;
template <typename T>
cudaError_t launch_get_clique_noalloc(const T* calib_clique, const CliqueOut& co, double* out_dev, cudaStream_t s);

// The paper's per-message kernels (Algorithm 1) with index-mapping tables,
// for comparison (jt_propagate_per_message): marginalise a clique onto a
// separator through its mapping table (snew, and the total into *sigma);
// ratio and scatter into the neighbour (normalising by *sigma when asked);
// evidence per clique; a table normalised to total one (its total into
// *total); the stage totals the finalisation reads.
template <typename T>
cudaError_t launch_msg_marg(const T* phi, const int32_t* mu, int32_t L, int32_t S, int interleaved, double* snew,
                            double* sigma, cudaStream_t s);
template <typename T>
cudaError_t launch_msg_scatter(T* phi, const int32_t* mu, int32_t L, int32_t S, int interleaved,
                               const double* snew, T* sold, const double* sigma, int normalise, cudaStream_t s);
template <typename T>
cudaError_t launch_clique_evidence(T* phi, int64_t n, const int4* obs, int n_obs, cudaStream_t s);
template <typename T>
cudaError_t launch_table_normalise(T* phi, int64_t n, double* total, cudaStream_t s);
cudaError_t launch_pack_totals(const double* sigma, const int32_t* sep_size, int nc, const double* root_total,
                               double* sums, cudaStream_t s);

// Maximum dynamic shared memory per CTA the kernels may use on this device
// with `ctas_per_sm` resident CTAs per SM.
int32_t smem_budget(int device, int ctas_per_sm = 1);

}  // namespace jt

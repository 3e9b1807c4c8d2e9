/*
 * jt.h -- C ABI of the GB300 junction-tree belief-propagation library (libjt).
 *
 * The library computes every Hugin message of a full collect-then-distribute
 * propagation on the GPU: marginalise a clique onto its separator (Eq. 2),
 * form the new/old separator ratio with 0/0 := 0 (Eq. 3 and the rule stated
 * after it), and scatter-multiply that ratio into the neighbouring clique
 * (Eq. 1, Sec. 3).  The schedule is Algorithm 4: collect towards the root
 * (Algorithm 2), then distribute from it (Algorithm 3); independent cliques
 * of one tree depth run concurrently (the breadth-first traversal the paper
 * allows in Sec. 3.3).  Many evidence cases of one resident tree are
 * propagated together.
 *
 * Conventions shared by every entry point:
 *   - Every function returns a jt_status; nothing aborts or throws across
 *     the ABI.  jt_last_error() gives a human-readable reason for the last
 *     failure on the calling thread.
 *   - The caller owns every pointer it passes; the library copies what it
 *     needs before returning (except where an entry point says it enqueues
 *     an asynchronous copy).
 *   - A stream is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  It may be a stream owned by another framework
 *     (for example torch.cuda.current_stream().cuda_stream).
 *   - Table layout: a clique's table lists its variables in the order given
 *     in clique_vars; the first-listed variable is the most significant
 *     digit of the flat index and the last-listed varies fastest (the layout
 *     of Fig. 2: for {A,B,D}, B = 0 selects entries {0,1,4,5}).
 *   - A tree is used by one host thread at a time; different trees are
 *     independent.
 */
#ifndef JT_H_
#define JT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jt_tree_s* jt_tree; /* opaque; owned by the library until jt_free */

typedef enum {
  JT_OK = 0,
  JT_ERR_INVALID_ARG = 1,         /* bad pointer, size, id, or non-finite/negative potential */
  JT_ERR_NOT_A_JUNCTION_TREE = 2, /* not a tree rooted at 0, or running intersection fails */
  JT_ERR_OOM = 3,                 /* device (or pinned host) allocation failed */
  JT_ERR_ZERO_EVIDENCE = 4,       /* P(e) = 0 for the queried case: no posterior exists */
  JT_ERR_TIMEOUT = 5,             /* a bounded device-side wait gave up */
  JT_ERR_CUDA = 6,                /* any other CUDA runtime error (see jt_last_error) */
  JT_ERR_STATE = 7,               /* result queried before a propagation covered the case */
  JT_ERR_UNSUPPORTED = 8          /* valid input outside the library's limits (see jt_last_error) */
} jt_status;

typedef enum { JT_F32 = 0, JT_F64 = 1 } jt_dtype;

/* jt_tree_desc.flags */
#define JT_MATERIALIZE_CLIQUES 0x1u /* also write every calibrated clique table per case */

/* Limits (checked by jt_load_tree; JT_ERR_UNSUPPORTED beyond them). */
#define JT_MAX_CLIQUE_VARS 32       /* variables per clique */
#define JT_MAX_TABLE_ENTRIES 0x7FFFFFF0LL /* entries of one clique table */
#define JT_MAX_CARD 32767           /* states of one variable */

/*
 * A junction tree J = (T, Phi) (Sec. 2.1): cliques C_i with variable sets
 * X_i and potential tables phi_{X_i}; the separator of the edge between a
 * clique and its parent is the intersection of their variable sets.
 */
typedef struct {
  int32_t n_vars;               /* variables 0 .. n_vars-1; each must appear in some clique */
  const int32_t* card;          /* [n_vars] states per variable, 2 <= card <= JT_MAX_CARD */
  int32_t n_cliques;            /* >= 1 */
  const int64_t* clique_off;    /* [n_cliques+1] CSR offsets into clique_vars */
  const int32_t* clique_vars;   /* listed order = table order (first most significant) */
  const int32_t* parent;        /* [n_cliques] parent[0] = -1 (root = clique 0) */
  const void* potentials;       /* host; tables concatenated in clique order, >= 0, finite;
                                   NULL: every table starts at one (then jt_init_from_cpts) */
  jt_dtype potentials_dtype;    /* element type of `potentials` */
  jt_dtype compute;             /* arithmetic type on the device (JT_F32 or JT_F64) */
  int32_t max_cases;            /* evidence-case slots kept resident, >= 1 */
  uint32_t flags;               /* JT_MATERIALIZE_CLIQUES, ... */
} jt_tree_desc;

/*
 * Validate the tree (Sec. 2.1 structure; running intersection), plan the
 * device layout, and upload the potentials.  Each clique table is stored
 * with its variables re-ordered so that its parent-separator variables are
 * the most significant digits, in `compute` precision.  An FP32 tree whose
 * cardinalities are not all powers of two, with max_cases >= 16 and without
 * JT_MATERIALIZE_CLIQUES, also gets a device copy with every cardinality
 * raised to the next power of two (the added states have zero potential, so
 * every result is the tree's own); it costs at most 5x the tables' memory,
 * counted in jt_get_info's device_bytes.  `stream` orders the uploads; the
 * call returns after they complete.  All inputs are copied.
 * On failure *out is set to NULL and nothing is leaked.
 */
jt_status jt_load_tree(const jt_tree_desc* desc, void* stream, jt_tree* out);

/*
 * Replace the evidence of case `case_id` (0 <= case_id < max_cases):
 * n_obs (variable, state) pairs from host arrays; n_obs = 0 clears it.
 * A repeated variable, an out-of-range id or state is JT_ERR_INVALID_ARG.
 * Evidence enters every clique that holds the variable by zeroing the
 * disagreeing entries (applied on the fly inside the message kernels).
 */
jt_status jt_set_evidence(jt_tree t, int32_t case_id, int32_t n_obs,
                          const int32_t* vars, const int32_t* states);

/*
 * Dense evidence for cases first_case .. first_case+n_cases-1: `states` is
 * int16 [n_cases][n_vars], -1 = unobserved.  `on_device` = 0: host memory
 * (copied before return); 1: device memory (copied asynchronously on
 * `stream`; the caller keeps it alive until the stream reaches that point).
 * States are range-checked on the device during propagation; a bad state
 * marks that case JT_ERR_INVALID_ARG.
 */
jt_status jt_set_evidence_dense(jt_tree t, int32_t first_case, int32_t n_cases,
                                const int16_t* states, int32_t on_device, void* stream);

/*
 * Belief_Propagation (Algorithm 4) for cases first_case .. first_case+n_cases-1:
 * collect (Algorithm 2) then distribute (Algorithm 3), every message by
 * Eq. 1-3, all cases in one CUDA-graph launch.  Asynchronous: only enqueues
 * work on `stream`.  Per-message rescaling keeps FP32 in range; log Z(e) is
 * accumulated in FP64.
 * The first call for a given (first_case, n_cases) records the schedules
 * the tree supports, runs each on `stream` and keeps the fastest; that call
 * synchronises `stream`.  The schedules: the whole tree per CTA (trees of
 * up to 2^17 entries), 32 cases on the lanes of a warp (FP32, 16 cases or
 * more; over a copy of the tree with power-of-two cardinalities when its
 * own are not), blocks of 8 or 4 cases sharing each table read, and one
 * case per work item (a single case times only the first and the last).
 * Then, for the width kept, it scales the planner's block size per
 * clique-size class (tables of < 2^14, < 2^18 and more entries) by 2^shift
 * where a shift is at least 2% faster; later ranges of the same tree and
 * width reuse the shifts.  jt_get_schedule reports the outcome.
 * Environment variables, read when a range is first propagated:
 * JT_CASE_BLOCK=0, 1, 4, 8 or 32 fixes the width (0 and 32 fall back where
 * they do not apply); JT_BLOCK_TUNE=0 keeps the planner's block sizes;
 * JT_WAIT_LIMIT_MS sets the limit of the kernels' bounded waits (2000 ms).
 * JT_PAD_CARDS=0, read by jt_load_tree, builds no power-of-two copy.
 */
jt_status jt_propagate(jt_tree t, int32_t first_case, int32_t n_cases, void* stream);

/*
 * The propagation of jt_propagate, issued without a graph with CUDA events
 * around its kernels, for measurement.  Waits for completion and writes, in
 * milliseconds, launch_ms[0] = the propagation kernel (every collect and
 * distribute message) and launch_ms[1] = the finalisation (marginals and
 * log Z).  max_launches must be >= 2; *n_launches is always set.  Results are
 * the same as jt_propagate's.  With the environment variable JT_TRACE=<file>
 * it also records every work item's SM and timeline (global timer, ns) and
 * writes them to <file> as CSV; JT_DEBUG_PLAN=1 prints each newly recorded
 * schedule's stages to stderr.
 */
jt_status jt_profile_propagate(jt_tree t, int32_t first_case, int32_t n_cases, void* stream,
                               float* launch_ms, int32_t max_launches, int32_t* n_launches);

/*
 * P(X = x | e) for variable `var` of case `case_id`: writes card[var]
 * doubles to host `out`.  Synchronises the stream of the last propagation.
 * JT_ERR_ZERO_EVIDENCE if P(e) = 0 (out is then filled with NaN),
 * JT_ERR_STATE if no propagation covered the case since its evidence changed.
 */
jt_status jt_get_marginal(jt_tree t, int32_t case_id, int32_t var, double* out);

/*
 * log Z(e) = log sum_x prod_C phi_C(x_C) prod_{v in E} [x_v = e_v], the log
 * of P(e) when the potentials are a normalised Bayesian-network
 * factorisation.  Synchronises like jt_get_marginal; -INFINITY and
 * JT_ERR_ZERO_EVIDENCE when P(e) = 0.
 */
jt_status jt_log_evidence(jt_tree t, int32_t case_id, double* out);

/*
 * Bulk read-out for cases first_case .. first_case+n_cases-1.
 * jt_get_marginals: double [n_cases][sum_v card[v]], variable v at offset
 * sum_{u<v} card[u].  jt_get_log_evidence: double [n_cases].
 * jt_get_status: int32 [n_cases] per-case jt_status.
 * `on_device` = 0: `out` is host memory and the call synchronises `stream`;
 * 1: `out` is device memory and the copy is only enqueued on `stream`.
 */
jt_status jt_get_marginals(jt_tree t, int32_t first_case, int32_t n_cases, double* out,
                           int32_t on_device, void* stream);
jt_status jt_get_log_evidence(jt_tree t, int32_t first_case, int32_t n_cases, double* out,
                              int32_t on_device, void* stream);
jt_status jt_get_status(jt_tree t, int32_t first_case, int32_t n_cases, int32_t* out);

/*
 * Calibrated table of clique `clique` for case `case_id`, normalised to sum
 * to one (= P(x_C | e)), in the caller's listed variable order: writes the
 * clique's table size of doubles to host `out`.  Needs
 * JT_MATERIALIZE_CLIQUES at load (else JT_ERR_STATE).
 */
jt_status jt_get_clique(jt_tree t, int32_t case_id, int32_t clique, double* out);

/*
 * The calibrated table of jt_get_clique, written to DEVICE memory without
 * allocating anything: no cudaMalloc, cudaFree or allocating library call,
 * so callers that must not allocate device memory can use it -- code that
 * runs while another component owns the device's memory (a fixed-size
 * arena or pool handed out up front), or a latency-critical serving path
 * whose policy forbids allocation (an allocation can synchronise the device
 * or fail under memory pressure).  The paper has no counterpart; it is a
 * read-out variant of the library.
 *
 * `out_device`: clique-size doubles of device memory owned by the caller,
 * filled with P(x_C | e) in the caller's listed variable order.  The work is
 * enqueued on `stream` (ordered after the last propagation) and the call
 * returns without waiting; check jt_get_status for the case before using the
 * values.  The normalising sum goes through a scratch array that lives in
 * the library for as long as it is loaded (every GPU that loads the library
 * holds it): the first call on a device looks its address up, so make that
 * first call before any stream capture.  Every call shares that array:
 * calls whose work overlaps on the GPU (different streams, no ordering)
 * race and give wrong results.  Cliques of more than 4,194,304 entries are
 * rejected with JT_ERR_UNSUPPORTED; JT_ERR_STATE as jt_get_clique.
 */
jt_status jt_get_clique_noalloc(jt_tree t, int32_t case_id, int32_t clique, double* out_device, void* stream);

/*
 * The paper's own propagation, for comparison (not the library's fast
 * path): collect then distribute (Algorithms 2-4) for case `case_id`, every
 * message by the per-message kernel of Algorithm 1 (Sec. 3.2): one launch
 * pair per message, one thread per separator entry, gathering and
 * scattering through precomputed index-mapping tables (Fig. 3) in the
 * layout `layout`: 0 = naive (each separator entry's list contiguous),
 * 1 = interleaved (the m-th elements of all lists adjacent; Sec. 4.5,
 * Fig. 8).  Collect messages are normalised by their totals (log Z
 * accumulates in FP64).  The tables are built on the host on first use of a
 * layout (one int32 per clique entry per incident separator) and kept until
 * jt_free.  Needs JT_MATERIALIZE_CLIQUES at load: it works in the case's
 * calibrated tables, which jt_get_clique then reads; the case's marginals
 * and log Z are then as after jt_propagate.  Synchronises `stream`;
 * `kernel_ms` (may be null) receives the device time of the whole
 * propagation.  JT_ERR_INVALID_ARG: bad case, layout or evidence state;
 * JT_ERR_STATE: loaded without JT_MATERIALIZE_CLIQUES.
 */
jt_status jt_propagate_per_message(jt_tree t, int32_t case_id, int32_t layout, void* stream, float* kernel_ms);

/*
 * Conditional probability tables of a Bayesian network over the tree's
 * variables, for jt_init_from_cpts.  CPT i is a table over its family
 * fam_vars[fam_off[i] .. fam_off[i+1]) (for P(v | pa(v)) the family is v and
 * its parents, in any order), laid out like a clique table: the
 * first-listed variable is the most significant digit.  Any non-negative
 * table over variables that share a clique is accepted; nothing requires
 * the columns to sum to one.
 */
typedef struct {
  int32_t n_cpts;
  const int32_t* fam_off;       /* [n_cpts+1] offsets into fam_vars, fam_off[0] = 0 */
  const int32_t* fam_vars;      /* families, each non-empty, no variable twice */
  const double* values;         /* host; tables concatenated in CPT order, >= 0, finite */
  const int32_t* home;          /* [n_cpts] clique that receives each CPT (it must hold the
                                   family), or NULL: the clique with the fewest entries that
                                   holds the family, ties to the lowest clique index */
} jt_cpt_desc;

/*
 * The Initialization step of Algorithm 4 (Sec. 3.3), on the device: every
 * clique table of the loaded tree is overwritten with the product of the
 * CPTs assigned to it, in ascending CPT order (one where a clique receives
 * none), computed in the tree's compute precision straight into the
 * resident table layout.  Together with separators that start at one, the
 * tree then represents the network's joint distribution.  Evidence slots are
 * kept, but every case must be propagated again before its results are read
 * (JT_ERR_STATE until then).  Work is enqueued on `stream` and the call
 * returns after it completes; `kernel_ms` (may be null) receives the device
 * time of the initialisation kernel.  All inputs are copied.
 * JT_ERR_INVALID_ARG: a null array, an empty or repeating family, a variable
 * id out of range, a negative or non-finite value, a family that no clique
 * (or not the named home clique) holds; the tables are then unchanged.
 */
jt_status jt_init_from_cpts(jt_tree t, const jt_cpt_desc* cpts, void* stream, float* kernel_ms);

/*
 * The resident (uncalibrated) table of clique `clique` -- as loaded, or as
 * jt_init_from_cpts built it -- in the caller's listed variable order and
 * compute precision widened to double: writes the clique's table size of
 * doubles to host `out`.  Synchronises with the tree's last stream.
 */
jt_status jt_get_potential(jt_tree t, int32_t clique, double* out);

/* Sizes and schedule facts of a loaded tree. */
typedef struct {
  int32_t n_vars, n_cliques, depth;  /* depth = largest clique depth (root 0) */
  int64_t entries;                   /* sum of clique table sizes */
  int64_t work_per_case;             /* sum over the 2(n-1) messages of |phi_src| + |phi_dst| (Eq. 4 numerator) */
  int64_t marginal_len;              /* sum_v card[v] */
  int64_t device_bytes;              /* device memory held by the tree */
  int64_t case_bytes;                /* of which per evidence-case slot (messages, evidence, results) */
  int32_t max_cases;
  jt_dtype compute;
  uint32_t flags;
} jt_tree_info;

jt_status jt_get_info(jt_tree t, jt_tree_info* out);

/* The schedule a propagation of the case range [first, first + n) uses
 * (recorded, and for several cases chosen by timing, on the range's first
 * jt_propagate).  Not part of the paper's method: it reports how the
 * library laid out the work (Sec. 3.4's per-message launches become one
 * persistent launch over work items).  JT_ERR_STATE if the range has not been
 * propagated yet; JT_ERR_INVALID_ARG for a bad range or a null `out`. */
typedef struct {
  int32_t case_block;   /* evidence cases per work item: 1, 4, 8, or 32 (one case per lane); 0: the whole
                           tree per CTA (a case is one CTA's work, from its shared memory) */
  int32_t n_items;      /* work items of one propagation */
  int32_t grid;         /* CTAs of the persistent launch */
  int32_t smem_bytes;   /* dynamic shared memory per CTA */
  int32_t window_entries; /* largest per-case window set of a work item */
  int32_t padded;       /* 1: the schedule runs over a copy of the tree with every cardinality raised to a
                           power of two (the added states impossible: zero potential), which case lanes
                           need; results are the original tree's */
  int8_t block_shift[4];  /* the block-size target of each clique-size class (tables of < 2^14, < 2^18 and
                             more entries; the 4th is unused) scaled by 2^shift, as the first timed range
                             of this width found fastest (0: the planner's own target) */
  int32_t reserved;
  float candidate_ms[5];  /* device time of one propagation of the range with 32, 8, 4 and 1 cases per
                             work item and with the whole tree per CTA, as the first use timed them
                             (-1: not timed or not applicable) */
} jt_schedule_info;

jt_status jt_get_schedule(jt_tree t, int32_t first, int32_t n, jt_schedule_info* out);

/* jt_propagate holding at most `max_ctas` SMs (0 or >= the SM count: all of
 * them).  The persistent propagation kernel claims one SM per CTA, so a
 * propagation of one tree normally holds the whole GPU; with a limit, the
 * propagations of several trees (each on its own stream) run side by side on
 * disjoint SMs, which is how a server overlaps batches of different trees.
 * Not part of the paper's method (its propagation is one kernel launch per
 * message, Sec. 3.4).  Results are the same as jt_propagate's (every
 * schedule computes Eq. 1-3 over Algorithms 2-4); the graph of each
 * (range, limit) is recorded on first use.  Errors as jt_propagate, plus
 * JT_ERR_INVALID_ARG for a negative limit. */
jt_status jt_propagate_ctas(jt_tree t, int32_t first, int32_t n, int32_t max_ctas, void* stream);

/* Start and end, on the GPU's global nanosecond timer, of the tree's most
 * recent propagation kernel (first CTA start, last CTA end): spans of
 * different trees' kernels are comparable, so a caller can tell whether two
 * propagations ran at the same time.  Synchronises with the tree's last
 * stream.  JT_ERR_STATE before the first propagation; JT_ERR_INVALID_ARG for
 * null outputs. */
jt_status jt_get_kernel_span(jt_tree t, uint64_t* start_ns, uint64_t* end_ns);

/* Release every resource of the tree (waits for its pending work). NULL is a no-op. */
void jt_free(jt_tree t);

/* Static string for a status code. */
const char* jt_strerror(jt_status s);

/* Reason for the last failing call on this thread ("" if none). */
const char* jt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* JT_H_ */

// C ABI of libjt: tree lifetime, evidence, propagation (one CUDA graph per
// case range: zeroing, the persistent propagation kernel, finalisation) and
// read-out.  See include/jt.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <memory>
#include <string>
#include <type_traits>
#include <vector>

#include "jt_internal.h"
#include "jt_init.h"
#include "jt_kernels.h"

using namespace jt;

namespace {

thread_local std::string g_err;

jt_status fail(jt_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

jt_status cuda_fail(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) return fail(JT_ERR_OOM, std::string(where) + ": out of device memory");
  return fail(JT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CU(call, where)                                 \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

constexpr int kCaseBlock = 8;   // evidence cases per work item when a propagation covers several cases

// A propagation shape (case range) recorded as a CUDA graph, with the device
// copy of its schedule.
struct GraphEntry {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  Schedule sched;
  std::vector<void*> dev_bufs;
  const DevStage* stages = nullptr;
  const DevPort* ports = nullptr;
  const DevField* fields = nullptr;
  const DevPos* pos = nullptr;
  const int32_t* deps = nullptr;
  const uint4* blobs = nullptr;
  const DevItem* items = nullptr;
  int32_t grid = 0, smem = 0;
  uint64_t wait_ns = 2000000000ull;  // limit of the kernel's bounded waits
  cudaEvent_t done = nullptr;   // recorded after every launch of the graph
  float candidate_ms[5] = {-1.f, -1.f, -1.f, -1.f, -1.f};   // first-use timing of widths 32, 8, 4, 1, whole tree
  bool padded = false;          // runs over the tree's power-of-two padded plan
  // whole-tree schedules: the level plan on the device
  const uint4* small_blobs = nullptr;
  const int32_t* small_idx = nullptr;   // packed level indices (SmallPlan::idx)
};

// State of the paper-literal per-message propagation (jt_propagate_per_message),
// built on first use: the index-mapping tables of every separator, on both of
// its sides, in one layout, and the scratch of the separator updates.
struct PerMsg {
  int layout = -1;
  std::vector<void*> bufs;                  // every device buffer below
  std::vector<const int32_t*> mu_child;     // [c]: entries of clique c per entry of its parent separator
  std::vector<const int32_t*> mu_parent;    // [c]: entries of the parent of c per entry of that separator
  double* snew = nullptr;                   // [msg_total] the message being sent
  void* sold = nullptr;                     // [msg_total] separator tables (element type)
  void* ones = nullptr;                     // [msg_total] ones, their start value
  double* sigma = nullptr;                  // [n_cliques + 2]: collect totals, root total, scratch
  int4* obs = nullptr;                      // [sum of clique sizes] evidence of every clique
  VarSrc* vs = nullptr;                     // marginal sources in the calibrated tables
};

}  // namespace

struct jt_tree_s {
  Plan plan;
  int device = 0;
  int n_sm = 0;
  int32_t smem_max = 0;
  jt_dtype compute = JT_F32;
  uint32_t flags = 0;
  int32_t max_cases = 1;
  size_t elem = 4;
  // device memory
  void* base = nullptr;           // permuted clique tables
  void* d_msg = nullptr;          // [max_cases][msg_stride] u | delta | joint
  double* d_sums = nullptr;       // [max_cases][2 n_cliques] stage totals
  int32_t* d_done = nullptr;      // [0] work queue, then [2 n_cliques][case blocks] finished blocks
  int32_t* d_err = nullptr;       // set by a kernel whose bounded wait gave up
  int32_t* d_status = nullptr;    // [max_cases]
  double* d_marg = nullptr;       // [max_cases][marg_total]
  double* d_logz = nullptr;       // [max_cases]
  int16_t* d_ev = nullptr;        // [max_cases][n_vars]
  void* d_calib = nullptr;        // [max_cases][base_len] (JT_MATERIALIZE_CLIQUES)
  double* d_scratch = nullptr;    // read-out scratch (partial sums + clique table)
  int64_t scratch_len = 0;
  int64_t scratch_parts = 0;      // leading partial-sum slots of the scratch
  VarSrc* d_vs = nullptr;         // marginal sources, joint layout 0 (one-case schedules)
  VarSrc* d_vs_fine = nullptr;    // joint layout 1 (case-block schedules)
  VarSrc* d_vs_var = nullptr;     // joint layout 2 (case-lane schedules: a joint per private variable)
  int32_t* d_order_var = nullptr;  // case-lane finalisation order of layout 2 (small sources first)
  int32_t n_small_var = 0;
  int32_t* d_sep_size = nullptr;
  int64_t device_bytes = 0;
  // host state
  int16_t* h_ev = nullptr;        // pinned mirror [max_cases][n_vars]
  std::vector<uint8_t> dirty;     // host mirror row newer than the device row
  std::vector<uint8_t> ready;     // a propagation covered the case since its evidence changed
  cudaEvent_t upload_done = nullptr;
  cudaEvent_t readout_ready = nullptr;  // orders the allocation-free read-out after a propagation
  cudaEvent_t readout_done = nullptr;   // recorded after an allocation-free read-out on its stream
  bool readout_pending = false;         // a later call that rewrites the tables must wait for it
  cudaEvent_t order_ev = nullptr;       // orders work on a new stream after the tree's last stream
  cudaStream_t cap_stream = nullptr;
  cudaStream_t last_stream = nullptr;
  std::map<std::tuple<int, int, int>, GraphEntry> graphs;   // (first case, cases, CTA cap; 0 = every SM)
  // block-target shifts per clique-size class found by the first timed range
  // of each (width, padded) schedule, reused by later ranges
  std::map<std::pair<int, bool>, std::array<int8_t, kBlockClasses>> tuned;
  unsigned long long* d_span = nullptr;   // [2] global-timer span of the last propagation kernel
  std::unique_ptr<PerMsg> permsg;
  // Power-of-two padded twin of the plan (FP32 trees with other
  // cardinalities): its own resident tables, derived from `base` on the
  // device, and its marginal sources and separator sizes; the case-lane
  // schedules of such a tree run over it.
  std::unique_ptr<Plan> pad;
  float* pad_base = nullptr;
  VarSrc* d_vs_pad = nullptr;
  int32_t* d_order_pad = nullptr;
  int32_t n_small_pad = 0;
  int32_t* d_sep_size_pad = nullptr;
  int4* d_pad_digits = nullptr;
  PadClique* d_pad_cliques = nullptr;
  int64_t pad_max = 0;                  // largest padded table
};

namespace {

template <typename T>
jt_status alloc(jt_tree t, T** p, int64_t n, const char* what) {
  *p = nullptr;
  if (n <= 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, (size_t)n * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, what);
  t->device_bytes += n * (int64_t)sizeof(T);
  return JT_OK;
}

void free_graphs(jt_tree t) {
  for (auto& kv : t->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    if (kv.second.done) cudaEventDestroy(kv.second.done);
    for (void* p : kv.second.dev_bufs) cudaFree(p);
  }
  t->graphs.clear();
}

void destroy(jt_tree t) {
  if (!t) return;
  cudaSetDevice(t->device);
  cudaDeviceSynchronize();
  free_graphs(t);
  if (t->permsg)
    for (void* q : t->permsg->bufs) cudaFree(q);
  void* ptrs[] = {t->base,   t->d_msg,  t->d_sums,  t->d_done,    t->d_err, t->d_status, t->d_marg,
                  t->d_logz, t->d_ev,   t->d_calib, t->d_scratch, t->d_vs,  t->d_vs_fine, t->d_vs_var, t->d_sep_size,
                  t->d_span, t->pad_base, t->d_vs_pad, t->d_sep_size_pad, t->d_pad_digits, t->d_pad_cliques,
                  t->d_order_var, t->d_order_pad};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (t->h_ev) cudaFreeHost(t->h_ev);
  if (t->upload_done) cudaEventDestroy(t->upload_done);
  if (t->readout_ready) cudaEventDestroy(t->readout_ready);
  if (t->readout_done) cudaEventDestroy(t->readout_done);
  if (t->order_ev) cudaEventDestroy(t->order_ev);
  if (t->cap_stream) cudaStreamDestroy(t->cap_stream);
  delete t;
}

template <typename V>
jt_status upload_vec(jt_tree t, std::vector<void*>* owner, const V** dst, const std::vector<V>& src,
                     const char* what) {
  V* p = nullptr;
  const size_t n = std::max<size_t>(1, src.size());
  cudaError_t e = cudaMalloc((void**)&p, n * sizeof(V));
  if (e != cudaSuccess) return cuda_fail(e, what);
  owner->push_back(p);
  if (!src.empty()) CU(cudaMemcpy(p, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice), what);
  *dst = p;
  (void)t;
  return JT_OK;
}

// Enqueue a whole propagation of a case range on `s`: zero the per-case
// accumulators, counters and the work queue, run the persistent propagation
// kernel, finalise.  With `ev` non-null an event is recorded before the
// propagation kernel, between it and the finalisation, and after.
template <typename T>
cudaError_t enqueue_schedule(jt_tree t, int case0, int n_cases, const GraphEntry& ge, cudaStream_t s,
                             cudaEvent_t* ev, uint64_t* trace = nullptr) {
  const Plan& p = ge.padded ? *t->pad : t->plan;
  const Schedule& sc = ge.sched;
  cudaError_t err = cudaSuccess;
  auto chk = [&](cudaError_t e) {
    if (err == cudaSuccess && e != cudaSuccess) err = e;
  };
  // (the whole-tree kernel writes each case's row, totals and status itself)
  const bool whole = sc.cb == kWholeTree;
  const int64_t msg_rows = sc.cb == kCaseLanes ? (int64_t)sc.n_cb * kCaseLanes : n_cases;
  if (!whole) {
    chk(cudaMemsetAsync((T*)t->d_msg + (int64_t)case0 * p.msg_stride, 0,
                        (size_t)msg_rows * p.msg_stride * sizeof(T), s));
    chk(cudaMemsetAsync(t->d_sums + (int64_t)case0 * 2 * p.n_cliques, 0,
                        (size_t)n_cases * 2 * p.n_cliques * sizeof(double), s));
    chk(cudaMemsetAsync(t->d_status + case0, 0, (size_t)n_cases * sizeof(int32_t), s));
    chk(cudaMemsetAsync(t->d_done, 0, (1 + 2ull * p.n_cliques * sc.n_cb) * sizeof(int32_t), s));
  }
  // the error word reports this propagation (a timed-out one leaves nothing
  // behind: every accumulator above starts again from zero)
  chk(cudaMemsetAsync(t->d_err, 0, sizeof(int32_t), s));
  // kernel span: start = min over CTAs (from all ones), end = max (from zero)
  chk(cudaMemsetAsync(t->d_span, 0xFF, sizeof(unsigned long long), s));
  chk(cudaMemsetAsync(t->d_span + 1, 0, sizeof(unsigned long long), s));
  PropArgs<T> a{};
  a.base = ge.padded ? (const T*)t->pad_base : (const T*)t->base;
  a.stages = ge.stages;
  a.ports = ge.ports;
  a.fields = ge.fields;
  a.pos = ge.pos;
  a.deps = ge.deps;
  a.blobs = ge.blobs;
  a.items = ge.items;
  a.n_items = (int32_t)sc.items.size();
  a.case0 = case0;
  a.n_cases = n_cases;
  a.n_cb = sc.n_cb;
  a.ev = t->d_ev;
  a.n_vars = p.n_vars;
  a.msg = (T*)t->d_msg;
  a.msg_stride = p.msg_stride;
  a.delta_off = p.msg_total;
  a.sums = t->d_sums;
  a.n_cliques = p.n_cliques;
  a.status = t->d_status;
  a.queue = t->d_done;
  a.done = t->d_done + 1;
  a.err = t->d_err;
  a.wait_ns = ge.wait_ns;
  a.calib = (T*)t->d_calib;
  a.calib_stride = p.base_len;
  a.trace = trace;
  a.span = t->d_span;
  a.ring = sc.ring;
  a.chunk = sc.chunk;
  a.max_k = sc.max_k;
  a.max_ports = sc.max_ports;
  a.max_fields = sc.max_fields;
  a.win_max = sc.win_max;
  a.blob_max = sc.blob_max;
  if (ev) chk(cudaEventRecord(ev[0], s));
  if (sc.cb == kWholeTree) {
    SmallArgs<T> w{};
    w.base = (const T*)t->base;
    w.blobs = ge.small_blobs;
    w.lv_blob_max = sc.small.lv_blob_max;
    w.idx = ge.small_idx;
    w.idx_len = (int32_t)sc.small.idx.size();
    w.o_seg_lv = sc.small.o_seg_lv;
    w.o_lv_stage_off = sc.small.o_lv_stage_off;
    w.o_stage_blob = sc.small.o_stage_blob;
    w.o_lv_stage = sc.small.o_lv_stage;
    w.o_sep_size = sc.small.o_sep_size;
    w.o_segs = sc.small.o_segs;
    w.idx_in_smem = sc.small.idx_in_smem ? 1 : 0;
    w.levels = sc.small.levels;
    w.ev = t->d_ev;
    w.n_vars = p.n_vars;
    w.msg = (T*)t->d_msg;
    w.msg_stride = p.msg_stride;
    w.msg_total = p.msg_total;
    w.sums = t->d_sums;
    w.n_cliques = p.n_cliques;
    w.status = t->d_status;
    w.case0 = case0;
    w.n_cases = n_cases;
    w.span = t->d_span;
    w.base_in_smem = sc.small.base_in_smem ? 1 : 0;
    w.base_len = p.base_len;
    w.desc_resident = sc.small.desc_resident ? 1 : 0;
    w.trace = trace;
    chk(launch_small<T>(w, ge.grid, ge.smem, s));
  } else if constexpr (std::is_same<T, float>::value) {
    if (sc.cb == kCaseLanes) chk(launch_propagate_cl(a, ge.grid, ge.smem, ge.padded, s));
    else chk(launch_propagate<T>(a, sc.cb, ge.grid, ge.smem, s));
  } else {
    chk(launch_propagate<T>(a, sc.cb, ge.grid, ge.smem, s));
  }
  if (ev) chk(cudaEventRecord(ev[1], s));
  FinalArgs<T> f{};
  // the joint layout the schedule's ports write
  f.vs = ge.padded ? t->d_vs_pad : sc.cb == kCaseLanes ? t->d_vs_var : (sc.cb > 1 ? t->d_vs_fine : t->d_vs);
  f.n_vars = p.n_vars;
  f.n_cliques = p.n_cliques;
  f.case0 = case0;
  f.n_cases = n_cases;
  f.msg = (const T*)t->d_msg;
  f.msg_stride = p.msg_stride;
  f.sums = t->d_sums;
  f.sep_size = ge.padded ? t->d_sep_size_pad : t->d_sep_size;
  f.status = t->d_status;
  f.marg_total = p.marg_total;
  f.marg_out = t->d_marg;
  f.logz_out = t->d_logz;
  f.lanes = sc.cb == kCaseLanes ? kCaseLanes : 1;
  f.var_order = ge.padded ? t->d_order_pad : t->d_order_var;
  f.n_small = ge.padded ? t->n_small_pad : t->n_small_var;
  if constexpr (std::is_same<T, float>::value) {
    if (sc.cb == kCaseLanes) chk(launch_finalize_cl(f, s));
    else chk(launch_finalize<T>(f, s));
  } else {
    chk(launch_finalize<T>(f, s));
  }
  if (ev) chk(cudaEventRecord(ev[2], s));
  return err;
}

// Plan the schedule of a case range, upload it, and record the propagation
// into a CUDA graph.
template <typename T>
jt_status record_schedule(jt_tree t, int case0, int n_cases, int cb, int cap, cudaStream_t s, GraphEntry* ge,
                          const int8_t* block_shift = nullptr) {
  std::string err;
  const int smem_cap = smem_budget(t->device, ctas_per_sm_for(cb)) - 256;
  const int sms = cap > 0 ? std::min(cap, t->n_sm) : t->n_sm;   // the SMs this propagation may hold
  // case lanes need power-of-two cliques: other trees run them padded
  ge->padded = cb == kCaseLanes && t->pad != nullptr;
  const Plan& plan = ge->padded ? *t->pad : t->plan;
  jt_status st = cb == kWholeTree
                     ? build_small_schedule(plan, (int)t->elem, n_cases, sms, smem_cap, &ge->sched, &err)
                     : build_schedule(plan, (int)t->elem, cb, n_cases, sms, smem_cap, &ge->sched, &err, block_shift);
  if (st != JT_OK) return fail(st, err);
  // Failure-path hooks, read when a range's graph is recorded (host-side
  // fault injection: nothing on the device faults or waits without limit).
  // JT_WAIT_LIMIT_MS sets the limit of every bounded device wait (2000 by
  // default); JT_FAULT_UNMET_DEPENDENCY=1 makes the first dependency of the
  // schedule wait for one block more than its stage has, so the waiting item
  // gives up at the limit and the propagation reports JT_ERR_TIMEOUT.
  if (const char* w = std::getenv("JT_WAIT_LIMIT_MS"); w && *w) {
    const long ms = std::strtol(w, nullptr, 10);
    if (ms > 0 && ms <= 60000) ge->wait_ns = (uint64_t)ms * 1000000ull;
  }
  if (const char* f = std::getenv("JT_FAULT_UNMET_DEPENDENCY"); f && *f == '1' && ge->sched.deps.size() >= 2)
    ge->sched.deps[1] += 1;
  const Schedule& sc = ge->sched;
  if ((st = upload_vec(t, &ge->dev_bufs, &ge->stages, sc.stages, "schedule upload")) != JT_OK) return st;
  if ((st = upload_vec(t, &ge->dev_bufs, &ge->ports, sc.ports, "schedule upload")) != JT_OK) return st;
  if ((st = upload_vec(t, &ge->dev_bufs, &ge->fields, sc.fields, "schedule upload")) != JT_OK) return st;
  if ((st = upload_vec(t, &ge->dev_bufs, &ge->pos, sc.pos, "schedule upload")) != JT_OK) return st;
  if ((st = upload_vec(t, &ge->dev_bufs, &ge->deps, sc.deps, "schedule upload")) != JT_OK) return st;
  if ((st = upload_vec(t, &ge->dev_bufs, &ge->blobs, sc.blobs, "schedule upload")) != JT_OK) return st;
  if ((st = upload_vec(t, &ge->dev_bufs, &ge->items, sc.items, "schedule upload")) != JT_OK) return st;
  ge->smem = prop_smem_bytes(sc, (int)t->elem);
  ge->grid = (int32_t)std::min<int64_t>((int64_t)sc.items.size(), (int64_t)sms * ctas_per_sm_for(cb));
  if (cb == kWholeTree) {
    const auto& sp = sc.small;
    if ((st = upload_vec(t, &ge->dev_bufs, &ge->small_blobs, sp.blobs, "schedule upload")) != JT_OK) return st;
    if ((st = upload_vec(t, &ge->dev_bufs, &ge->small_idx, sp.idx, "schedule upload")) != JT_OK) return st;
    ge->smem = sp.smem;
    // every case is one CTA's work; a CTA of 1024 threads at 64 registers
    // fills an SM's register file, so one per SM is resident
    ge->grid = (int32_t)std::min<int64_t>(n_cases, (int64_t)sms);
  }
  if (const char* dbg = std::getenv("JT_DEBUG_PLAN"); dbg && *dbg == '1') {
    std::fprintf(stderr, "[jt plan] cases=%d cb=%d n_cb=%d items=%zu grid=%d smem=%d ring=%d win_max=%d\n", n_cases,
                 sc.cb, sc.n_cb, sc.items.size(), ge->grid, ge->smem, sc.ring, sc.win_max);
    for (const DevStage& S : sc.stages) {
      if (S.n_blocks == 0) continue;
      std::fprintf(stderr, "  stage c=%d pass=%d n=%d B=%d blocks=%d bits=%d kin=%d ports=%d(in %d) win=%d deps=%d\n",
                   S.clique, S.pass, S.n, S.B, S.n_blocks, S.bits, S.kin, S.np, S.nin, S.win_len, S.ndep);
    }
  }
  CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t e = enqueue_schedule<T>(t, case0, n_cases, *ge, s, nullptr);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e, "recording the propagation");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
  ge->graph = g;
  CU(cudaGraphInstantiate(&ge->exec, g, 0), "graph instantiate");
  return JT_OK;
}

void drop_graph(GraphEntry& ge) {
  if (ge.exec) cudaGraphExecDestroy(ge.exec);
  if (ge.graph) cudaGraphDestroy(ge.graph);
  if (ge.done) cudaEventDestroy(ge.done);
  for (void* p : ge.dev_bufs) cudaFree(p);
  ge.exec = nullptr;
  ge.graph = nullptr;
  ge.done = nullptr;
  ge.dev_bufs.clear();
}

// Device time of one launch of a recorded propagation on `s` (ms), or a
// negative value on error.
float time_graph(const GraphEntry& ge, cudaStream_t s);

// The fastest of `reps` launches (after the caller's warm-up): block-size
// candidates differ by a few percent, below one launch's spread.
float time_graph_min(const GraphEntry& ge, cudaStream_t s, int reps) {
  float best = -1.f;
  for (int r = 0; r < reps; ++r) {
    const float ms = time_graph(ge, s);
    if (ms >= 0.f && (best < 0.f || ms < best)) best = ms;
  }
  return best;
}

float time_graph(const GraphEntry& ge, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = -1.f;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
      cudaEventRecord(e0, s) == cudaSuccess && cudaGraphLaunch(ge.exec, s) == cudaSuccess &&
      cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess)
    cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return ms;
}

// The propagation graph of a case range, recorded on first use.  Several
// cases can go one per work item (more, shorter items; every item streams
// its table for one case), in blocks of 4 or kCaseBlock = 8 (each streamed
// table chunk serves the block's cases), or, for FP32 trees of power-of-two
// cliques, kCaseLanes = 32 cases on the lanes of every warp.  Which is
// fastest depends on the tree and the number of cases, so the first use of a
// multi-case range times each schedule the tree supports once (after a
// warm-up launch of each; the launches compute the same propagation the
// caller asked for) and keeps the fastest.  JT_CASE_BLOCK=1, 4, 8 or 32 in
// the environment fixes the choice instead (32 falls back to 8 where case
// lanes do not apply).
jt_status get_graph(jt_tree t, int first, int n, int cap, cudaStream_t s, GraphEntry** out) {
  auto key = std::make_tuple(first, n, cap);
  auto it = t->graphs.find(key);
  if (it == t->graphs.end()) {
    if (t->graphs.size() >= 64) {
      // every cached graph's last launch has finished before it is destroyed
      for (auto& kv : t->graphs)
        if (kv.second.done) CU(cudaEventSynchronize(kv.second.done), "graph cache eviction");
      free_graphs(t);
    }
    int forced = -1;
    if (const char* f = std::getenv("JT_CASE_BLOCK"); f && *f) {
      const std::string v(f);
      if (v == "0" || v == "1" || v == "4" || v == "8" || v == "32") forced = std::stoi(v);
    }
    auto record = [&](int cb, GraphEntry* ge, const int8_t* shift = nullptr) {
      return t->compute == JT_F64 ? record_schedule<double>(t, first, n, cb, cap, t->cap_stream, ge, shift)
                                  : record_schedule<float>(t, first, n, cb, cap, t->cap_stream, ge, shift);
    };
    std::vector<int> cands;
    if (forced == kWholeTree) {
      cands = {kWholeTree, n == 1 ? 1 : kCaseBlock};  // the first one the tree supports
    } else if (n == 1) {
      cands = forced == 1 ? std::vector<int>{1} : std::vector<int>{kWholeTree, 1};
    } else if (forced == kCaseLanes) {
      cands = {kCaseLanes, kCaseBlock};
    } else if (forced > 0) {
      cands = {forced};
    } else {
      cands.push_back(kWholeTree);
      if (t->compute == JT_F32 && n >= 16) cands.push_back(kCaseLanes);
      cands.push_back(kCaseBlock);
      if (n > 4) cands.push_back(4);
      cands.push_back(1);
    }
    const bool timed_choice = forced < 0;
    float timed[5] = {-1.f, -1.f, -1.f, -1.f, -1.f};
    GraphEntry best;
    bool have = false;
    float best_ms = -1.f;
    jt_status first_err = JT_OK;
    std::string first_msg;
    for (int cb : cands) {
      GraphEntry ge;
      const jt_status st = record(cb, &ge);
      if (st != JT_OK) {
        drop_graph(ge);
        if (const char* dbg = std::getenv("JT_DEBUG_PLAN"); dbg && *dbg == '1')
          std::fprintf(stderr, "[jt plan] cases=%d width %d not used: %s\n", n, cb, g_err.c_str());
        if (first_err == JT_OK) {
          first_err = st;
          first_msg = g_err;
        }
        continue;
      }
      if (!timed_choice) {
        std::swap(best, ge);
        have = true;
        break;
      }
      time_graph(ge, s);
      const float ms = time_graph(ge, s);
      timed[cb == kCaseLanes ? 0 : cb == kCaseBlock ? 1 : cb == 4 ? 2 : cb == 1 ? 3 : 4] = ms;
      if (!have || (ms >= 0.f && (best_ms < 0.f || ms < best_ms))) {
        std::swap(best, ge);
        best_ms = ms;
        have = true;
      }
      drop_graph(ge);
    }
    if (!have) return fail(first_err == JT_OK ? JT_ERR_CUDA : first_err, first_msg);
    // Block sizes per clique-size class for the chosen width: from an
    // earlier range of this tree and width, or searched here one class at a
    // time (the block target halved, then doubled, and a direction that
    // helps once more; a change is kept when it is at least 2% faster).
    // JT_BLOCK_TUNE=0 keeps the planner's targets.
    const char* bt = std::getenv("JT_BLOCK_TUNE");
    if (best.sched.cb != kWholeTree && !(bt && *bt == '0')) {
      const auto tkey = std::make_pair(best.sched.cb, best.padded);
      auto tit = t->tuned.find(tkey);
      if (tit != t->tuned.end()) {
        bool zero = true;
        for (int8_t x : tit->second) zero = zero && x == 0;
        GraphEntry ge;
        if (!zero && record(best.sched.cb, &ge, tit->second.data()) == JT_OK) {
          drop_graph(best);
          std::swap(best, ge);
        }
        drop_graph(ge);
      } else if (timed_choice) {
        bool present[kBlockClasses] = {};
        for (const DevStage& S : best.sched.stages)
          if (S.n_blocks > 0) present[block_class(S.n)] = true;
        std::array<int8_t, kBlockClasses> cur{};
        const float cur_ms0 = time_graph_min(best, s, 3);
        float cur_ms = cur_ms0 >= 0.f ? cur_ms0 : best_ms;
        auto attempt = [&](int q, int8_t v) {
          std::array<int8_t, kBlockClasses> trial = cur;
          trial[q] = v;
          GraphEntry ge;
          bool kept = false;
          if (record(best.sched.cb, &ge, trial.data()) == JT_OK) {
            time_graph(ge, s);
            const float ms = time_graph_min(ge, s, 3);
            if (ms >= 0.f && ms < 0.98f * cur_ms) {
              std::swap(best, ge);
              cur = trial;
              cur_ms = ms;
              kept = true;
            }
          }
          drop_graph(ge);
          return kept;
        };
        for (int q = 0; q < kBlockClasses; ++q) {
          if (!present[q]) continue;
          // halved, then doubled; a direction that helps is tried once more
          for (int8_t d : {(int8_t)-1, (int8_t)1})
            if (attempt(q, d)) {
              attempt(q, (int8_t)(2 * d));
              break;
            }
        }
        t->tuned[tkey] = cur;
      }
    }
    CU(cudaEventCreateWithFlags(&best.done, cudaEventDisableTiming), "event");
    std::copy(timed, timed + 5, best.candidate_ms);
    it = t->graphs.emplace(key, std::move(best)).first;
  }
  *out = &it->second;
  return JT_OK;
}

jt_status check_tree(jt_tree t) {
  if (!t) return fail(JT_ERR_INVALID_ARG, "null tree");
  cudaError_t e = cudaSetDevice(t->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return JT_OK;
}

jt_status check_range(jt_tree t, int32_t first, int32_t n) {
  if (first < 0 || n < 0 || (int64_t)first + n > t->max_cases)
    return fail(JT_ERR_INVALID_ARG, "case range outside [0, max_cases)");
  return JT_OK;
}

jt_status wait_upload(jt_tree t) {
  CU(cudaEventSynchronize(t->upload_done), "waiting for evidence upload");
  return JT_OK;
}

jt_status sync_last(jt_tree t) {
  CU(cudaStreamSynchronize(t->last_stream), "synchronising the propagation stream");
  return JT_OK;
}

// Order work about to be enqueued on `s` after the tree's earlier work: the
// tree's last stream (work on two streams would otherwise run at the same
// time over the same per-tree buffers), and an allocation-free read-out that
// may still be reading a calibrated table on a stream of its own.
jt_status order_on(jt_tree t, cudaStream_t s) {
  if (s != t->last_stream) {
    CU(cudaEventRecord(t->order_ev, t->last_stream), "stream ordering");
    CU(cudaStreamWaitEvent(s, t->order_ev, 0), "stream ordering");
  }
  if (t->readout_pending) {
    CU(cudaStreamWaitEvent(s, t->readout_done, 0), "read-out ordering");
    t->readout_pending = false;
  }
  return JT_OK;
}

// A kernel gave up a bounded wait: every result since is invalid.
jt_status check_err(jt_tree t) {
  int32_t e = 0;
  CU(cudaMemcpy(&e, t->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost), "error word read");
  if (e) return fail(JT_ERR_TIMEOUT, "a device-side wait timed out; results are invalid");
  return JT_OK;
}

jt_status case_status(jt_tree t, int32_t cs, int32_t* code) {
  jt_status es = check_err(t);
  if (es != JT_OK) return es;
  int32_t st = 0;
  CU(cudaMemcpy(&st, t->d_status + cs, sizeof(int32_t), cudaMemcpyDeviceToHost), "status read");
  if (st & kStatusBadState) *code = JT_ERR_INVALID_ARG;
  else if (st & kStatusZero) *code = JT_ERR_ZERO_EVIDENCE;
  else *code = JT_OK;
  return JT_OK;
}

template <typename T>
jt_status load_typed(jt_tree t, const jt_tree_desc* d, cudaStream_t s) {
  Plan& p = t->plan;
  std::vector<T> host((size_t)p.base_len);
  permute_tables<T>(p, d->potentials, d->potentials_dtype, host.data());
  jt_status st;
  if ((st = alloc(t, (T**)&t->base, p.base_len, "clique tables")) != JT_OK) return st;
  CU(cudaMemcpyAsync(t->base, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, s), "table upload");
  // (case-lane schedules keep whole slabs of kCaseLanes cases: the last slab of
  // a range may reach past max_cases)
  const int64_t msg_stride = std::max<int64_t>(p.msg_stride, t->pad ? t->pad->msg_stride : 0);
  if ((st = alloc(t, (T**)&t->d_msg, msg_stride * (t->max_cases + kCaseLanes - 1), "per-case messages")) != JT_OK)
    return st;
  if (t->flags & JT_MATERIALIZE_CLIQUES) {
    if ((st = alloc(t, (T**)&t->d_calib, p.base_len * t->max_cases, "calibrated tables")) != JT_OK) return st;
  }
  CU(cudaStreamSynchronize(s), "table upload");
  return JT_OK;
}

// A power-of-two padded twin pays where case lanes run (FP32, batches of
// cases) on a tree with other cardinalities.  JT_PAD_CARDS=0 turns it off.
bool want_pad(const Plan& p, const jt_tree_desc* d) {
  if (d->compute != JT_F32 || (d->flags & JT_MATERIALIZE_CLIQUES) || d->max_cases < 16) return false;
  if (const char* e = std::getenv("JT_PAD_CARDS"); e && *e == '0') return false;
  return std::any_of(p.pow2.begin(), p.pow2.end(), [](uint8_t x) { return x == 0; });
}

// Device side of the padded twin: its tables (from the resident ones), the
// map that derives them, its marginal sources and separator sizes.
jt_status load_pad(jt_tree t, cudaStream_t s) {
  const Plan& q = *t->pad;
  jt_status st;
  if ((st = alloc(t, &t->pad_base, q.base_len, "padded tables")) != JT_OK) return st;
  CU(cudaMemsetAsync(t->pad_base, 0, (size_t)q.base_len * sizeof(float), s), "padded tables");
  const PadMap m = build_pad_map(t->plan, q);
  if ((st = alloc(t, &t->d_pad_digits, (int64_t)m.digits.size(), "padding map")) != JT_OK) return st;
  if ((st = alloc(t, &t->d_pad_cliques, (int64_t)m.cliques.size(), "padding map")) != JT_OK) return st;
  if ((st = alloc(t, &t->d_vs_pad, q.n_vars, "marginal sources")) != JT_OK) return st;
  if ((st = alloc(t, &t->d_sep_size_pad, q.n_cliques, "separator sizes")) != JT_OK) return st;
  CU(cudaMemcpy(t->d_pad_digits, m.digits.data(), m.digits.size() * sizeof(int4), cudaMemcpyHostToDevice),
     "descriptor upload");
  CU(cudaMemcpy(t->d_pad_cliques, m.cliques.data(), m.cliques.size() * sizeof(PadClique), cudaMemcpyHostToDevice),
     "descriptor upload");
  CU(cudaMemcpy(t->d_vs_pad, q.vsrc[2].data(), q.n_vars * sizeof(VarSrc), cudaMemcpyHostToDevice),
     "descriptor upload");
  {
    const std::vector<int32_t> order = fin_order(q.vsrc[2], &t->n_small_pad);
    if ((st = alloc(t, &t->d_order_pad, q.n_vars, "finalisation order")) != JT_OK) return st;
    CU(cudaMemcpy(t->d_order_pad, order.data(), q.n_vars * sizeof(int32_t), cudaMemcpyHostToDevice),
       "descriptor upload");
  }
  CU(cudaMemcpy(t->d_sep_size_pad, q.sep_size.data(), q.n_cliques * sizeof(int32_t), cudaMemcpyHostToDevice),
     "descriptor upload");
  for (const PadClique& c : m.cliques) t->pad_max = std::max(t->pad_max, c.n_pad);
  CU(launch_pad_tables((const float*)t->base, t->pad_base, t->d_pad_digits, t->d_pad_cliques, t->plan.n_cliques,
                       t->pad_max, s),
     "padding the tables");
  return JT_OK;
}

// Upload the evidence rows of [first, first+n) that changed on the host, as
// contiguous runs from the pinned mirror.
jt_status upload_dirty(jt_tree t, int first, int n, cudaStream_t s) {
  const int nv = t->plan.n_vars;
  bool uploaded = false;
  for (int i = first; i < first + n;) {
    if (!t->dirty[i]) {
      ++i;
      continue;
    }
    int j = i;
    while (j < first + n && t->dirty[j]) t->dirty[j++] = 0;
    CU(cudaMemcpyAsync(t->d_ev + (int64_t)i * nv, t->h_ev + (int64_t)i * nv, (size_t)(j - i) * nv * sizeof(int16_t),
                       cudaMemcpyHostToDevice, s), "evidence upload");
    uploaded = true;
    i = j;
  }
  if (uploaded) CU(cudaEventRecord(t->upload_done, s), "event");
  return JT_OK;
}

// Read-out geometry of a clique: listed cardinalities and the permuted stride
// of each listed position.
CliqueOut clique_out(const Plan& p, int clique) {
  CliqueOut co{};
  co.n = (int32_t)p.n_entries[clique];
  co.k = (int32_t)p.vars[clique].size();
  const auto& lv = p.vars[clique];
  const auto& pv = p.pvars[clique];
  std::vector<int64_t> pst(pv.size());
  int64_t s = 1;
  for (int i = (int)pv.size() - 1; i >= 0; --i) {
    pst[i] = s;
    s *= p.card[pv[i]];
  }
  for (int i = 0; i < co.k; ++i) {
    co.lcard[i] = p.card[lv[i]];
    for (int j = 0; j < co.k; ++j)
      if (pv[j] == lv[i]) co.pst[i] = (int32_t)pst[j];
  }
  return co;
}

}  // namespace

namespace {

// Index-mapping tables of the per-message propagation in `layout` (0 naive:
// entry j's list contiguous; 1 interleaved: the m-th elements of all lists
// adjacent), one per side of every separator, over the permuted tables.
jt_status build_permsg(jt_tree t, int layout) {
  const Plan& p = t->plan;
  const int nc = p.n_cliques;
  auto pm = std::make_unique<PerMsg>();
  pm->layout = layout;
  pm->mu_child.assign(nc, nullptr);
  pm->mu_parent.assign(nc, nullptr);
  auto dalloc = [&](size_t bytes, void** q, const char* what) -> jt_status {
    cudaError_t e = cudaMalloc(q, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return cuda_fail(e, what);
    pm->bufs.push_back(*q);
    return JT_OK;
  };
  auto release = [&]() {
    for (void* q : pm->bufs) cudaFree(q);
  };
  // strides of every variable in a clique's permuted table
  auto stride_of = [&](int q, int v) -> int64_t {
    const auto& pv = p.pvars[q];
    int64_t st = 1;
    for (int i = (int)pv.size() - 1; i >= 0; --i) {
      if (pv[i] == v) return st;
      st *= p.card[pv[i]];
    }
    return -1;
  };
  std::vector<int32_t> mu;
  for (int c = 1; c < nc; ++c) {
    const auto& sv = p.sep[c];
    const int32_t S = p.sep_size[c];
    for (int side = 0; side < 2; ++side) {
      const int q = side == 0 ? c : p.parent[c];
      const int64_t N = p.n_entries[q], L = N / S;
      std::vector<int64_t> st(sv.size());
      for (size_t i = 0; i < sv.size(); ++i) st[i] = stride_of(q, sv[i]);
      mu.assign((size_t)N, 0);
      std::vector<int32_t> cnt((size_t)S, 0);
      for (int64_t x = 0; x < N; ++x) {
        int64_t j = 0;
        for (size_t i = 0; i < sv.size(); ++i) j = j * p.card[sv[i]] + (x / st[i]) % p.card[sv[i]];
        const int64_t m = cnt[(size_t)j]++;
        mu[(size_t)(layout ? m * S + j : j * L + m)] = (int32_t)x;
      }
      void* d = nullptr;
      jt_status st2 = dalloc((size_t)N * sizeof(int32_t), &d, "mapping tables");
      if (st2 != JT_OK) {
        release();
        return st2;
      }
      if (cudaMemcpy(d, mu.data(), (size_t)N * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
        release();
        return fail(JT_ERR_CUDA, "mapping table upload");
      }
      (side == 0 ? pm->mu_child : pm->mu_parent)[c] = static_cast<const int32_t*>(d);
    }
  }
  const size_t mt = (size_t)std::max(1, p.msg_total);
  void* q = nullptr;
  jt_status st = JT_OK;
  if ((st = dalloc(mt * sizeof(double), &q, "separator scratch")) != JT_OK) return release(), st;
  pm->snew = static_cast<double*>(q);
  if ((st = dalloc(mt * t->elem, &pm->sold, "separator tables")) != JT_OK) return release(), st;
  if ((st = dalloc(mt * t->elem, &pm->ones, "separator start values")) != JT_OK) return release(), st;
  if ((st = dalloc((size_t)(nc + 2) * sizeof(double), &q, "message totals")) != JT_OK) return release(), st;
  pm->sigma = static_cast<double*>(q);
  size_t kk = 0;
  for (int c = 0; c < nc; ++c) kk += p.pvars[c].size();
  if ((st = dalloc(std::max<size_t>(kk, 1) * sizeof(int4), &q, "evidence lists")) != JT_OK) return release(), st;
  pm->obs = static_cast<int4*>(q);
  if ((st = dalloc((size_t)p.n_vars * sizeof(VarSrc), &q, "marginal sources")) != JT_OK) return release(), st;
  pm->vs = static_cast<VarSrc*>(q);
  // ones
  if (t->compute == JT_F64) {
    std::vector<double> o(mt, 1.0);
    if (cudaMemcpy(pm->ones, o.data(), mt * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
      return release(), fail(JT_ERR_CUDA, "upload");
  } else {
    std::vector<float> o(mt, 1.0f);
    if (cudaMemcpy(pm->ones, o.data(), mt * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      return release(), fail(JT_ERR_CUDA, "upload");
  }
  // every variable's marginal from the smallest calibrated clique holding it
  std::vector<VarSrc> vs((size_t)p.n_vars);
  for (int v = 0; v < p.n_vars; ++v) {
    int best = -1;
    for (int c = 0; c < nc; ++c)
      if (stride_of(c, v) > 0 && (best < 0 || p.n_entries[c] < p.n_entries[best])) best = c;
    VarSrc& r = vs[(size_t)v];
    r.card = p.card[v];
    r.card_out = p.card[v];
    r.moff = p.moff[v];
    r.off = (int32_t)p.base_off[best];
    r.size = (int32_t)p.n_entries[best];
    r.st = (int32_t)stride_of(best, v);
  }
  if (cudaMemcpy(pm->vs, vs.data(), vs.size() * sizeof(VarSrc), cudaMemcpyHostToDevice) != cudaSuccess)
    return release(), fail(JT_ERR_CUDA, "upload");
  if (t->permsg)
    for (void* b : t->permsg->bufs) cudaFree(b);
  t->permsg = std::move(pm);
  return JT_OK;
}

// Collect then distribute (Algorithms 2-4) for one case, one launch pair per
// message, into the case's calibrated tables.
template <typename T>
cudaError_t run_permsg(jt_tree t, int cs, const std::vector<int4>& obs, const std::vector<int>& obs_off,
                       cudaStream_t s) {
  const Plan& p = t->plan;
  const PerMsg& pm = *t->permsg;
  const int nc = p.n_cliques, lay = pm.layout;
  T* row = (T*)t->d_calib + (int64_t)cs * p.base_len;
  T* sold = (T*)pm.sold;
  cudaError_t err = cudaSuccess;
  auto chk = [&](cudaError_t e) {
    if (err == cudaSuccess && e != cudaSuccess) err = e;
  };
  chk(cudaMemcpyAsync(row, t->base, (size_t)p.base_len * sizeof(T), cudaMemcpyDeviceToDevice, s));
  chk(cudaMemcpyAsync(sold, pm.ones, (size_t)std::max(1, p.msg_total) * sizeof(T), cudaMemcpyDeviceToDevice, s));
  chk(cudaMemsetAsync(pm.sigma, 0, (size_t)(nc + 2) * sizeof(double), s));
  chk(cudaMemsetAsync(t->d_status + cs, 0, sizeof(int32_t), s));
  if (!obs.empty())
    chk(cudaMemcpyAsync(pm.obs, obs.data(), obs.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  for (int c = 0; c < nc; ++c)
    chk(launch_clique_evidence<T>(row + p.base_off[c], p.n_entries[c], pm.obs + obs_off[c],
                                  obs_off[c + 1] - obs_off[c], s));
  // collect: child to parent, deepest level first, each message normalised
  for (int dd = p.max_depth; dd >= 1; --dd)
    for (int c : p.levels[dd]) {
      const int q = p.parent[c];
      const int32_t S = p.sep_size[c];
      double* sn = pm.snew + p.sep_off[c];
      chk(launch_msg_marg<T>(row + p.base_off[c], pm.mu_child[c], (int32_t)(p.n_entries[c] / S), S, lay, sn,
                             pm.sigma + c, s));
      chk(launch_msg_scatter<T>(row + p.base_off[q], pm.mu_parent[c], (int32_t)(p.n_entries[q] / S), S, lay, sn,
                                sold + p.sep_off[c], pm.sigma + c, 1, s));
    }
  // the root normalised to total one (its total is the evidence's last factor)
  chk(launch_table_normalise<T>(row + p.base_off[0], p.n_entries[0], pm.sigma + nc, s));
  // distribute: parent to child, from the root
  for (int dd = 0; dd < p.max_depth; ++dd)
    for (int q : p.levels[dd])
      for (int c : p.children[q]) {
        const int32_t S = p.sep_size[c];
        double* sn = pm.snew + p.sep_off[c];
        chk(launch_msg_marg<T>(row + p.base_off[q], pm.mu_parent[c], (int32_t)(p.n_entries[q] / S), S, lay, sn,
                               pm.sigma + nc + 1, s));
        chk(launch_msg_scatter<T>(row + p.base_off[c], pm.mu_child[c], (int32_t)(p.n_entries[c] / S), S, lay, sn,
                                  sold + p.sep_off[c], pm.sigma + nc + 1, 0, s));
      }
  chk(launch_pack_totals(pm.sigma, t->d_sep_size, nc, pm.sigma + nc, t->d_sums + (int64_t)cs * 2 * nc, s));
  FinalArgs<T> f{};
  f.vs = pm.vs;
  f.n_vars = p.n_vars;
  f.n_cliques = nc;
  f.case0 = cs;
  f.n_cases = 1;
  f.msg = (const T*)t->d_calib;
  f.msg_stride = p.base_len;
  f.sums = t->d_sums;
  f.sep_size = t->d_sep_size;
  f.status = t->d_status;
  f.marg_total = p.marg_total;
  f.marg_out = t->d_marg;
  f.logz_out = t->d_logz;
  f.lanes = 1;
  chk(launch_finalize<T>(f, s));
  return err;
}

}  // namespace

namespace {

// Device buffers of one call, freed on every path out of it.
struct TempBufs {
  std::vector<void*> p;
  ~TempBufs() {
    for (void* x : p) cudaFree(x);
  }
  template <typename U>
  cudaError_t upload(U** d, const std::vector<U>& h, cudaStream_t s) {
    *d = nullptr;
    if (h.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)d, h.size() * sizeof(U));
    if (e != cudaSuccess) return e;
    p.push_back(*d);
    return cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(U), cudaMemcpyHostToDevice, s);
  }
};

// Multiplier and shifts of UDiv for a divisor 1 <= d < 2^31.
UDiv make_udiv(uint32_t d) {
  uint32_t l = 0;
  while ((uint64_t{1} << l) < d) ++l;
  const uint64_t mul = ((uint64_t{1} << 32) * ((uint64_t{1} << l) - d)) / d + 1;
  return UDiv{(uint32_t)mul, (uint16_t)std::min<uint32_t>(l, 1), (uint16_t)(l > 0 ? l - 1 : 0)};
}

int32_t log2_exact(int64_t x) {
  int32_t r = 0;
  while ((int64_t{1} << r) < x) ++r;
  return r;
}

template <typename T>
jt_status init_typed(jt_tree t, const std::vector<InitItem>& items, const std::vector<InitClique>& cl,
                     const std::vector<InitFactor>& fac, const std::vector<InitTerm>& terms,
                     const std::vector<double>& values, cudaStream_t s, float* kernel_ms) {
  std::vector<T> vals(values.begin(), values.end());
  TempBufs tb;
  InitItem* d_items;
  InitClique* d_cl;
  InitFactor* d_fac;
  InitTerm* d_terms;
  T* d_vals;
  CU(tb.upload(&d_items, items, s), "initialisation upload");
  CU(tb.upload(&d_cl, cl, s), "initialisation upload");
  CU(tb.upload(&d_fac, fac, s), "initialisation upload");
  CU(tb.upload(&d_terms, terms, s), "initialisation upload");
  CU(tb.upload(&d_vals, vals, s), "initialisation upload");
  // (events created here are destroyed on every path out)
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaSuccess;
  if (kernel_ms) {
    e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
  }
  if (e == cudaSuccess)
    e = launch_init_cliques<T>((T*)t->base, d_items, (int32_t)items.size(), d_cl, d_fac, d_terms, d_vals, t->n_sm, s);
  if (e == cudaSuccess && kernel_ms) e = cudaEventRecord(ev[1], s);
  // the padded twin follows the new tables
  if (e == cudaSuccess && t->pad)
    e = launch_pad_tables((const float*)t->base, t->pad_base, t->d_pad_digits, t->d_pad_cliques, t->plan.n_cliques,
                          t->pad_max, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && kernel_ms) e = cudaEventElapsedTime(kernel_ms, ev[0], ev[1]);
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (e != cudaSuccess) return cuda_fail(e, "clique initialisation");
  return JT_OK;
}

}  // namespace

extern "C" {

const char* jt_strerror(jt_status s) {
  switch (s) {
    case JT_OK: return "ok";
    case JT_ERR_INVALID_ARG: return "invalid argument";
    case JT_ERR_NOT_A_JUNCTION_TREE: return "not a junction tree";
    case JT_ERR_OOM: return "out of memory";
    case JT_ERR_ZERO_EVIDENCE: return "evidence has probability zero";
    case JT_ERR_TIMEOUT: return "device wait timed out";
    case JT_ERR_CUDA: return "CUDA error";
    case JT_ERR_STATE: return "result not available in this state";
    case JT_ERR_UNSUPPORTED: return "unsupported input";
  }
  return "unknown status";
}

const char* jt_last_error(void) { return g_err.c_str(); }

jt_status jt_load_tree(const jt_tree_desc* d, void* stream, jt_tree* out) {
  if (!out) return fail(JT_ERR_INVALID_ARG, "null output handle");
  *out = nullptr;
  g_err.clear();
  std::unique_ptr<jt_tree_s> t(new jt_tree_s());
  jt_status st = build_plan(d, &t->plan, &g_err);
  if (st != JT_OK) return st;
  t->compute = d->compute;
  t->flags = d->flags;
  t->max_cases = d->max_cases;
  t->elem = d->compute == JT_F64 ? 8 : 4;
  Plan& p = t->plan;
  if (want_pad(p, d)) {
    // padding multiplies the table entries: kept within a few times the tree
    auto q = std::make_unique<Plan>();
    std::string perr;
    if (build_padded_plan(p, q.get(), &perr) == JT_OK && q->base_len <= 5 * p.base_len &&
        q->base_len < (1ll << 31))
      t->pad = std::move(q);
  }
  int dev = 0;
  CU(cudaGetDevice(&dev), "cudaGetDevice");
  t->device = dev;
  CU(cudaDeviceGetAttribute(&t->n_sm, cudaDevAttrMultiProcessorCount, dev), "device query");
  t->smem_max = smem_budget(dev, 1);
  cudaStream_t s = (cudaStream_t)stream;
  jt_tree raw = t.release();
  auto bail = [&](jt_status code) {
    std::string keep = g_err;
    destroy(raw);
    g_err = keep;
    return code;
  };
  if ((st = (raw->compute == JT_F64 ? load_typed<double>(raw, d, s) : load_typed<float>(raw, d, s))) != JT_OK)
    return bail(st);
  if (raw->pad && (st = load_pad(raw, s)) != JT_OK) return bail(st);
  const int nc = p.n_cliques;
  if ((st = alloc(raw, &raw->d_sums, 2ll * nc * raw->max_cases, "stage totals")) != JT_OK) return bail(st);
  if ((st = alloc(raw, &raw->d_done, 1 + 2ll * nc * raw->max_cases, "block counters")) != JT_OK) return bail(st);
  if ((st = alloc(raw, &raw->d_err, 1, "error word")) != JT_OK) return bail(st);
  if ((st = alloc(raw, &raw->d_span, 2, "kernel span")) != JT_OK) return bail(st);
  if (cudaMemset(raw->d_span, 0, 2 * sizeof(unsigned long long)) != cudaSuccess)
    return bail(fail(JT_ERR_CUDA, "memset"));
  if (cudaMemset(raw->d_err, 0, sizeof(int32_t)) != cudaSuccess) return bail(fail(JT_ERR_CUDA, "memset"));
  if ((st = alloc(raw, &raw->d_status, raw->max_cases, "status")) != JT_OK) return bail(st);
  if (cudaMemset(raw->d_status, 0, raw->max_cases * sizeof(int32_t)) != cudaSuccess)
    return bail(fail(JT_ERR_CUDA, "memset"));
  if ((st = alloc(raw, &raw->d_marg, (int64_t)raw->max_cases * p.marg_total, "marginals")) != JT_OK) return bail(st);
  if ((st = alloc(raw, &raw->d_logz, raw->max_cases, "log evidence")) != JT_OK) return bail(st);
  const int64_t nev = (int64_t)raw->max_cases * p.n_vars;
  if ((st = alloc(raw, &raw->d_ev, nev, "evidence")) != JT_OK) return bail(st);
  if (cudaMemset(raw->d_ev, 0xFF, nev * sizeof(int16_t)) != cudaSuccess) return bail(fail(JT_ERR_CUDA, "memset"));
  if ((st = alloc(raw, &raw->d_vs, p.n_vars, "marginal sources")) != JT_OK) return bail(st);
  if (cudaMemcpy(raw->d_vs, p.vsrc[0].data(), p.n_vars * sizeof(VarSrc), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(fail(JT_ERR_CUDA, "descriptor upload"));
  if ((st = alloc(raw, &raw->d_vs_var, p.n_vars, "marginal sources")) != JT_OK) return bail(st);
  if (cudaMemcpy(raw->d_vs_var, p.vsrc[2].data(), p.n_vars * sizeof(VarSrc), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(fail(JT_ERR_CUDA, "descriptor upload"));
  {
    const std::vector<int32_t> order = fin_order(p.vsrc[2], &raw->n_small_var);
    if ((st = alloc(raw, &raw->d_order_var, p.n_vars, "finalisation order")) != JT_OK) return bail(st);
    if (cudaMemcpy(raw->d_order_var, order.data(), p.n_vars * sizeof(int32_t), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return bail(fail(JT_ERR_CUDA, "descriptor upload"));
  }
  if ((st = alloc(raw, &raw->d_vs_fine, p.n_vars, "marginal sources")) != JT_OK) return bail(st);
  if (cudaMemcpy(raw->d_vs_fine, p.vsrc[1].data(), p.n_vars * sizeof(VarSrc), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return bail(fail(JT_ERR_CUDA, "descriptor upload"));
  if ((st = alloc(raw, &raw->d_sep_size, nc, "separator sizes")) != JT_OK) return bail(st);
  if (cudaMemcpy(raw->d_sep_size, p.sep_size.data(), nc * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(fail(JT_ERR_CUDA, "descriptor upload"));
  int64_t maxn = 0;
  for (int64_t n : p.n_entries) maxn = std::max(maxn, n);
  // [partial sums of the normalisation, 16-byte aligned] [clique table]
  raw->scratch_parts = ((maxn + kNoAllocPerBlock - 1) / kNoAllocPerBlock + 1) / 2 * 2;
  raw->scratch_len = raw->scratch_parts + maxn + 2;
  if ((st = alloc(raw, &raw->d_scratch, raw->scratch_len, "read-out scratch")) != JT_OK) return bail(st);
  cudaError_t e = cudaMallocHost((void**)&raw->h_ev, (size_t)nev * sizeof(int16_t));
  if (e != cudaSuccess) return bail(cuda_fail(e, "pinned evidence mirror"));
  std::fill(raw->h_ev, raw->h_ev + nev, (int16_t)-1);
  raw->dirty.assign(raw->max_cases, 0);
  raw->ready.assign(raw->max_cases, 0);
  if ((e = cudaEventCreateWithFlags(&raw->upload_done, cudaEventDisableTiming)) != cudaSuccess)
    return bail(cuda_fail(e, "event"));
  if ((e = cudaEventRecord(raw->upload_done, s)) != cudaSuccess) return bail(cuda_fail(e, "event"));
  if ((e = cudaEventCreateWithFlags(&raw->readout_ready, cudaEventDisableTiming)) != cudaSuccess)
    return bail(cuda_fail(e, "event"));
  if ((e = cudaEventCreateWithFlags(&raw->readout_done, cudaEventDisableTiming)) != cudaSuccess)
    return bail(cuda_fail(e, "event"));
  if ((e = cudaEventCreateWithFlags(&raw->order_ev, cudaEventDisableTiming)) != cudaSuccess)
    return bail(cuda_fail(e, "event"));
  if ((e = cudaStreamCreateWithFlags(&raw->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(cuda_fail(e, "stream"));
  raw->last_stream = s;
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(cuda_fail(e, "load"));
  *out = raw;
  return JT_OK;
}

jt_status jt_set_evidence(jt_tree t, int32_t case_id, int32_t n_obs, const int32_t* vars, const int32_t* states) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  if (case_id < 0 || case_id >= t->max_cases) return fail(JT_ERR_INVALID_ARG, "case_id out of range");
  if (n_obs < 0 || (n_obs > 0 && (!vars || !states))) return fail(JT_ERR_INVALID_ARG, "bad observation arrays");
  const int nv = t->plan.n_vars;
  std::vector<int16_t> row(nv, -1);
  for (int i = 0; i < n_obs; ++i) {
    const int v = vars[i], s = states[i];
    if (v < 0 || v >= nv) return fail(JT_ERR_INVALID_ARG, "observed variable id out of range");
    if (s < 0 || s >= t->plan.card[v]) return fail(JT_ERR_INVALID_ARG, "observed state out of range");
    if (row[v] >= 0) return fail(JT_ERR_INVALID_ARG, "variable observed twice");
    row[v] = (int16_t)s;
  }
  if ((st = wait_upload(t)) != JT_OK) return st;
  std::memcpy(t->h_ev + (int64_t)case_id * nv, row.data(), nv * sizeof(int16_t));
  t->dirty[case_id] = 1;
  t->ready[case_id] = 0;
  return JT_OK;
}

jt_status jt_set_evidence_dense(jt_tree t, int32_t first, int32_t n, const int16_t* states, int32_t on_device,
                                void* stream) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  if ((st = check_range(t, first, n)) != JT_OK) return st;
  if (n == 0) return JT_OK;
  if (!states) return fail(JT_ERR_INVALID_ARG, "null states");
  const int nv = t->plan.n_vars;
  const size_t bytes = (size_t)n * nv * sizeof(int16_t);
  if (on_device) {
    if ((st = order_on(t, (cudaStream_t)stream)) != JT_OK) return st;
    CU(cudaMemcpyAsync(t->d_ev + (int64_t)first * nv, states, bytes, cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream), "evidence copy");
    for (int i = 0; i < n; ++i) {
      t->dirty[first + i] = 0;
      t->ready[first + i] = 0;
    }
    return JT_OK;
  }
  for (int64_t i = 0; i < (int64_t)n * nv; ++i) {
    const int s = states[i];
    if (s < -1 || s >= t->plan.card[i % nv]) return fail(JT_ERR_INVALID_ARG, "observed state out of range");
  }
  if ((st = wait_upload(t)) != JT_OK) return st;
  std::memcpy(t->h_ev + (int64_t)first * nv, states, bytes);
  for (int i = 0; i < n; ++i) {
    t->dirty[first + i] = 1;
    t->ready[first + i] = 0;
  }
  return JT_OK;
}

jt_status jt_propagate(jt_tree t, int32_t first, int32_t n, void* stream) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  if ((st = check_range(t, first, n)) != JT_OK) return st;
  if (n == 0) return JT_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = order_on(t, s)) != JT_OK) return st;
  if ((st = upload_dirty(t, first, n, s)) != JT_OK) return st;
  GraphEntry* ge = nullptr;
  if ((st = get_graph(t, first, n, 0, s, &ge)) != JT_OK) return st;
  CU(cudaGraphLaunch(ge->exec, s), "graph launch");
  CU(cudaEventRecord(ge->done, s), "event");
  for (int i = first; i < first + n; ++i) t->ready[i] = 1;
  t->last_stream = s;
  return JT_OK;
}

jt_status jt_propagate_ctas(jt_tree t, int32_t first, int32_t n, int32_t max_ctas, void* stream) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  if ((st = check_range(t, first, n)) != JT_OK) return st;
  if (max_ctas < 0) return fail(JT_ERR_INVALID_ARG, "negative CTA limit");
  if (n == 0) return JT_OK;
  const int cap = (max_ctas == 0 || max_ctas >= t->n_sm) ? 0 : max_ctas;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = order_on(t, s)) != JT_OK) return st;
  if ((st = upload_dirty(t, first, n, s)) != JT_OK) return st;
  GraphEntry* ge = nullptr;
  if ((st = get_graph(t, first, n, cap, s, &ge)) != JT_OK) return st;
  CU(cudaGraphLaunch(ge->exec, s), "graph launch");
  CU(cudaEventRecord(ge->done, s), "event");
  for (int i = first; i < first + n; ++i) t->ready[i] = 1;
  t->last_stream = s;
  return JT_OK;
}

jt_status jt_get_kernel_span(jt_tree t, uint64_t* start_ns, uint64_t* end_ns) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  if (!start_ns || !end_ns) return fail(JT_ERR_INVALID_ARG, "null output");
  if ((st = sync_last(t)) != JT_OK) return st;
  unsigned long long h[2] = {0, 0};
  CU(cudaMemcpy(h, t->d_span, sizeof(h), cudaMemcpyDeviceToHost), "span read");
  if (h[1] == 0 || h[0] > h[1]) return fail(JT_ERR_STATE, "no propagation kernel has run");
  *start_ns = h[0];
  *end_ns = h[1];
  return JT_OK;
}

jt_status jt_profile_propagate(jt_tree t, int32_t first, int32_t n, void* stream, float* launch_ms,
                               int32_t max_launches, int32_t* n_launches) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  if ((st = check_range(t, first, n)) != JT_OK) return st;
  const int nl = 2;
  if (n_launches) *n_launches = nl;
  if (n == 0) return JT_OK;
  if (!launch_ms || max_launches < nl) return fail(JT_ERR_INVALID_ARG, "launch_ms needs 2 slots");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = order_on(t, s)) != JT_OK) return st;
  if ((st = upload_dirty(t, first, n, s)) != JT_OK) return st;
  GraphEntry* ge = nullptr;
  if ((st = get_graph(t, first, n, 0, s, &ge)) != JT_OK) return st;
  // JT_TRACE=<file>: also record every work item's SM and timeline
  // (global timer, ns) and write them to <file> as CSV
  const char* trace_path = std::getenv("JT_TRACE");
  uint64_t* trace = nullptr;
  const size_t n_items = ge->sched.items.size();
  if (trace_path && *trace_path) {
    CU(cudaMalloc((void**)&trace, n_items * kTraceSlots * sizeof(uint64_t)), "trace buffer");
    CU(cudaMemset(trace, 0, n_items * kTraceSlots * sizeof(uint64_t)), "trace buffer");
  }
  std::vector<cudaEvent_t> ev(nl + 1, nullptr);
  for (auto& e : ev) CU(cudaEventCreate(&e), "event");
  cudaError_t err = t->compute == JT_F64 ? enqueue_schedule<double>(t, first, n, *ge, s, ev.data(), trace)
                                         : enqueue_schedule<float>(t, first, n, *ge, s, ev.data(), trace);
  if (err == cudaSuccess) err = cudaEventSynchronize(ev[nl]);
  for (int i = 0; i < nl && err == cudaSuccess; ++i) err = cudaEventElapsedTime(&launch_ms[i], ev[i], ev[i + 1]);
  for (auto& e : ev) cudaEventDestroy(e);
  if (trace) {
    std::vector<uint64_t> h(n_items * kTraceSlots);
    if (err == cudaSuccess) err = cudaMemcpy(h.data(), trace, h.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost);
    cudaFree(trace);
    FILE* f = err == cudaSuccess ? std::fopen(trace_path, "w") : nullptr;
    if (f != nullptr && ge->sched.cb == kWholeTree) {
      // phase ends per level of the first case (ns from the kernel start)
      std::fprintf(f, "level,start_ns,ratios_ns,segments_ns,scales_ns\n");
      std::fprintf(f, "-1,0,0,%lld,%lld\n", (long long)(h[1] - h[0]), (long long)(h[1] - h[0]));
      for (int lv = 0; lv < ge->sched.small.levels; ++lv)
        std::fprintf(f, "%d,%lld,%lld,%lld,%lld\n", lv, (long long)(h[2 + 4 * lv] - h[0]),
                     (long long)(h[3 + 4 * lv] - h[0]), (long long)(h[4 + 4 * lv] - h[0]),
                     (long long)(h[5 + 4 * lv] - h[0]));
      std::fclose(f);
      f = nullptr;
    }
    if (f != nullptr) {
      uint64_t t0 = ~0ull;
      for (size_t i = 0; i < n_items; ++i)
        if (h[i * kTraceSlots + 1]) t0 = std::min(t0, h[i * kTraceSlots + 1]);
      std::fprintf(f, "item,stage,clique,pass,block,cbk,n,sm,start_ns,prepared_ns,stream_ns,streamed_ns,done_ns,"
                      "chunk_wait_ns,claimed_ns,issued_ns,published_ns,deps_met_ns,prep_start_ns\n");
      for (size_t i = 0; i < n_items; ++i) {
        const DevItem& w = ge->sched.items[i];
        const DevStage& S = ge->sched.stages[w.stage];
        const uint64_t* r = &h[i * kTraceSlots];
        std::fprintf(f, "%zu,%d,%d,%d,%d,%d,%d,%llu,%lld,%lld,%lld,%lld,%lld,%lld,%lld,%lld,%lld,%lld,%lld\n", i,
                     w.stage, S.clique, S.pass, w.block, w.cbk, w.n, (unsigned long long)r[0], (long long)(r[1] - t0),
                     (long long)(r[2] - t0), (long long)(r[3] - t0), (long long)(r[4] - t0), (long long)(r[5] - t0),
                     (long long)r[6], (long long)(r[7] - t0), (long long)(r[8] - t0), (long long)(r[9] - t0),
                     (long long)(r[10] - t0), (long long)(r[11] - t0));
      }
      std::fclose(f);
    }
  }
  if (err != cudaSuccess) return cuda_fail(err, "profiled propagation");
  for (int i = first; i < first + n; ++i) t->ready[i] = 1;
  t->last_stream = s;
  return JT_OK;
}

jt_status jt_get_marginal(jt_tree t, int32_t case_id, int32_t var, double* out) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  if (case_id < 0 || case_id >= t->max_cases) return fail(JT_ERR_INVALID_ARG, "case_id out of range");
  if (var < 0 || var >= t->plan.n_vars || !out) return fail(JT_ERR_INVALID_ARG, "bad variable or output");
  if (!t->ready[case_id]) return fail(JT_ERR_STATE, "case not propagated since its evidence changed");
  if ((st = sync_last(t)) != JT_OK) return st;
  const int kc = t->plan.card[var];
  CU(cudaMemcpy(out, t->d_marg + (int64_t)case_id * t->plan.marg_total + t->plan.moff[var], kc * sizeof(double),
                cudaMemcpyDeviceToHost), "marginal read");
  int32_t code = 0;
  if ((st = case_status(t, case_id, &code)) != JT_OK) return st;
  if (code != JT_OK) {
    for (int i = 0; i < kc; ++i) out[i] = NAN;
    return fail((jt_status)code, code == JT_ERR_ZERO_EVIDENCE ? "P(e) = 0" : "bad evidence state");
  }
  return JT_OK;
}

jt_status jt_log_evidence(jt_tree t, int32_t case_id, double* out) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  if (case_id < 0 || case_id >= t->max_cases || !out) return fail(JT_ERR_INVALID_ARG, "bad case or output");
  if (!t->ready[case_id]) return fail(JT_ERR_STATE, "case not propagated since its evidence changed");
  if ((st = sync_last(t)) != JT_OK) return st;
  CU(cudaMemcpy(out, t->d_logz + case_id, sizeof(double), cudaMemcpyDeviceToHost), "log evidence read");
  int32_t code = 0;
  if ((st = case_status(t, case_id, &code)) != JT_OK) return st;
  if (code == JT_ERR_ZERO_EVIDENCE) {
    *out = -INFINITY;
    return fail(JT_ERR_ZERO_EVIDENCE, "P(e) = 0");
  }
  if (code != JT_OK) return fail((jt_status)code, "bad evidence state");
  return JT_OK;
}

jt_status jt_get_marginals(jt_tree t, int32_t first, int32_t n, double* out, int32_t on_device, void* stream) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  if ((st = check_range(t, first, n)) != JT_OK) return st;
  if (n == 0) return JT_OK;
  if (!out) return fail(JT_ERR_INVALID_ARG, "null output");
  for (int i = first; i < first + n; ++i)
    if (!t->ready[i]) return fail(JT_ERR_STATE, "case not propagated since its evidence changed");
  const size_t bytes = (size_t)n * t->plan.marg_total * sizeof(double);
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaMemcpyAsync(out, t->d_marg + (int64_t)first * t->plan.marg_total, bytes,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s), "marginals read");
  if (!on_device) CU(cudaStreamSynchronize(s), "marginals read");
  return JT_OK;
}

jt_status jt_get_log_evidence(jt_tree t, int32_t first, int32_t n, double* out, int32_t on_device, void* stream) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  if ((st = check_range(t, first, n)) != JT_OK) return st;
  if (n == 0) return JT_OK;
  if (!out) return fail(JT_ERR_INVALID_ARG, "null output");
  for (int i = first; i < first + n; ++i)
    if (!t->ready[i]) return fail(JT_ERR_STATE, "case not propagated since its evidence changed");
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaMemcpyAsync(out, t->d_logz + first, (size_t)n * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s), "log evidence read");
  if (!on_device) CU(cudaStreamSynchronize(s), "log evidence read");
  return JT_OK;
}

jt_status jt_get_status(jt_tree t, int32_t first, int32_t n, int32_t* out) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  if ((st = check_range(t, first, n)) != JT_OK) return st;
  if (n == 0) return JT_OK;
  if (!out) return fail(JT_ERR_INVALID_ARG, "null output");
  if ((st = sync_last(t)) != JT_OK) return st;
  if ((st = check_err(t)) != JT_OK) return st;
  std::vector<int32_t> raw(n);
  CU(cudaMemcpy(raw.data(), t->d_status + first, n * sizeof(int32_t), cudaMemcpyDeviceToHost), "status read");
  for (int i = 0; i < n; ++i) {
    if (!t->ready[first + i]) out[i] = JT_ERR_STATE;
    else if (raw[i] & kStatusBadState) out[i] = JT_ERR_INVALID_ARG;
    else if (raw[i] & kStatusZero) out[i] = JT_ERR_ZERO_EVIDENCE;
    else out[i] = JT_OK;
  }
  return JT_OK;
}

jt_status jt_get_schedule(jt_tree t, int32_t first, int32_t n, jt_schedule_info* out) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  if ((st = check_range(t, first, n)) != JT_OK) return st;
  if (!out || n < 1) return fail(JT_ERR_INVALID_ARG, "null output or empty range");
  auto it = t->graphs.find(std::make_tuple(first, n, 0));
  if (it == t->graphs.end()) return fail(JT_ERR_STATE, "case range not propagated yet");
  const GraphEntry& ge = it->second;
  *out = jt_schedule_info{};
  out->case_block = ge.sched.cb;
  out->n_items = (int32_t)ge.sched.items.size();
  out->grid = ge.grid;
  out->smem_bytes = ge.smem;
  out->window_entries = ge.sched.win_max;
  out->padded = ge.padded ? 1 : 0;
  for (int q = 0; q < kBlockClasses; ++q) out->block_shift[q] = ge.sched.block_shift[q];
  std::copy(ge.candidate_ms, ge.candidate_ms + 5, out->candidate_ms);
  return JT_OK;
}

jt_status jt_get_clique(jt_tree t, int32_t case_id, int32_t clique, double* out) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  const Plan& p = t->plan;
  if (case_id < 0 || case_id >= t->max_cases || clique < 0 || clique >= p.n_cliques || !out)
    return fail(JT_ERR_INVALID_ARG, "bad case, clique or output");
  if (!(t->flags & JT_MATERIALIZE_CLIQUES)) return fail(JT_ERR_STATE, "tree loaded without JT_MATERIALIZE_CLIQUES");
  if (!t->ready[case_id]) return fail(JT_ERR_STATE, "case not propagated since its evidence changed");
  const CliqueOut co = clique_out(p, clique);
  cudaStream_t strm = t->last_stream;
  const int64_t off = (int64_t)case_id * p.base_len + p.base_off[clique];
  cudaError_t e = t->compute == JT_F64
                      ? launch_get_clique<double>((const double*)t->d_calib + off, co,
                                                  t->d_scratch + t->scratch_parts, t->d_scratch, strm)
                      : launch_get_clique<float>((const float*)t->d_calib + off, co,
                                                 t->d_scratch + t->scratch_parts, t->d_scratch, strm);
  if (e != cudaSuccess) return cuda_fail(e, "clique read-out");
  CU(cudaMemcpyAsync(out, t->d_scratch + t->scratch_parts, (size_t)co.n * sizeof(double), cudaMemcpyDeviceToHost,
                     strm),
     "clique read");
  CU(cudaStreamSynchronize(strm), "clique read");
  int32_t code = 0;
  if ((st = case_status(t, case_id, &code)) != JT_OK) return st;
  if (code != JT_OK) return fail((jt_status)code, "case has no posterior");
  return JT_OK;
}

jt_status jt_get_clique_noalloc(jt_tree t, int32_t case_id, int32_t clique, double* out_device, void* stream) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  const Plan& p = t->plan;
  if (case_id < 0 || case_id >= t->max_cases || clique < 0 || clique >= p.n_cliques || !out_device)
    return fail(JT_ERR_INVALID_ARG, "bad case, clique or output");
  if (p.n_entries[clique] > kNoAllocMaxEntries)
    return fail(JT_ERR_UNSUPPORTED, "clique has " + std::to_string(p.n_entries[clique]) +
                                        " entries; the allocation-free read-out handles at most " +
                                        std::to_string(kNoAllocMaxEntries));
  if (!(t->flags & JT_MATERIALIZE_CLIQUES)) return fail(JT_ERR_STATE, "tree loaded without JT_MATERIALIZE_CLIQUES");
  if (!t->ready[case_id]) return fail(JT_ERR_STATE, "case not propagated since its evidence changed");
  const CliqueOut co = clique_out(p, clique);
  cudaStream_t strm = (cudaStream_t)stream;
  if (strm != t->last_stream) {  // after the propagation that wrote the table (event made at load)
    CU(cudaEventRecord(t->readout_ready, t->last_stream), "read-out ordering");
    CU(cudaStreamWaitEvent(strm, t->readout_ready, 0), "read-out ordering");
  }
  const int64_t off = (int64_t)case_id * p.base_len + p.base_off[clique];
  cudaError_t e = t->compute == JT_F64
                      ? launch_get_clique_noalloc<double>((const double*)t->d_calib + off, co, out_device, strm)
                      : launch_get_clique_noalloc<float>((const float*)t->d_calib + off, co, out_device, strm);
  if (e != cudaSuccess) return cuda_fail(e, "allocation-free clique read-out");
  // a later propagation, per-message propagation or initialisation of this
  // tree waits for the read-out before it rewrites the table
  CU(cudaEventRecord(t->readout_done, strm), "read-out ordering");
  t->readout_pending = true;
  return JT_OK;
}

jt_status jt_init_from_cpts(jt_tree t, const jt_cpt_desc* cp, void* stream, float* kernel_ms) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  if (!cp || cp->n_cpts < 0) return fail(JT_ERR_INVALID_ARG, "null CPT descriptor or negative count");
  const int32_t n = cp->n_cpts;
  if (n > 0 && (!cp->fam_off || !cp->fam_vars || !cp->values)) return fail(JT_ERR_INVALID_ARG, "null CPT array");
  const Plan& p = t->plan;
  const int nc = p.n_cliques;
  // cliques holding each variable, ascending
  std::vector<std::vector<int32_t>> holders(p.n_vars);
  for (int c = 0; c < nc; ++c)
    for (int v : p.vars[c]) holders[v].push_back(c);
  auto position = [&](int c, int v) {  // permuted position of v in clique c, or -1
    const auto& pv = p.pvars[c];
    for (int i = 0; i < (int)pv.size(); ++i)
      if (pv[i] == v) return i;
    return -1;
  };
  std::vector<int32_t> home(n);
  std::vector<int64_t> val_off(n + 1, 0);
  std::vector<int32_t> seen(p.n_vars, -1);
  if (n > 0 && cp->fam_off[0] != 0) return fail(JT_ERR_INVALID_ARG, "fam_off[0] must be 0");
  for (int i = 0; i < n; ++i) {
    const int32_t a = cp->fam_off[i], b = cp->fam_off[i + 1];
    const std::string who = "CPT " + std::to_string(i);
    if (b <= a) return fail(JT_ERR_INVALID_ARG, who + " has an empty family");
    int64_t size = 1;
    for (int32_t j = a; j < b; ++j) {
      const int32_t v = cp->fam_vars[j];
      if (v < 0 || v >= p.n_vars) return fail(JT_ERR_INVALID_ARG, who + ": variable id out of range");
      if (seen[v] == i) return fail(JT_ERR_INVALID_ARG, who + ": a variable appears twice in its family");
      seen[v] = i;
      size *= p.card[v];
      if (size > JT_MAX_TABLE_ENTRIES) return fail(JT_ERR_INVALID_ARG, who + ": no clique holds its family");
    }
    auto holds = [&](int c) {
      for (int32_t j = a; j < b; ++j)
        if (position(c, cp->fam_vars[j]) < 0) return false;
      return true;
    };
    int32_t h = -1;
    if (cp->home) {
      h = cp->home[i];
      if (h < 0 || h >= nc) return fail(JT_ERR_INVALID_ARG, who + ": home clique out of range");
      if (!holds(h)) return fail(JT_ERR_INVALID_ARG, who + ": its home clique does not hold its family");
    } else {
      for (int32_t c : holders[cp->fam_vars[a]])
        if ((h < 0 || p.n_entries[c] < p.n_entries[h]) && holds(c)) h = c;
      if (h < 0) return fail(JT_ERR_INVALID_ARG, who + ": no clique holds its family");
    }
    home[i] = h;
    val_off[i + 1] = val_off[i] + size;
  }
  std::vector<double> values(cp->values, cp->values + val_off[n]);
  for (double x : values)
    if (!(x >= 0.0) || !std::isfinite(x)) return fail(JT_ERR_INVALID_ARG, "CPT values must be finite and >= 0");

  // descriptors: per clique its CPTs in ascending order, per CPT the
  // permuted stride and CPT stride of each family variable
  std::vector<std::vector<int32_t>> by_clique(nc);
  for (int i = 0; i < n; ++i) by_clique[home[i]].push_back(i);
  std::vector<InitClique> cl(nc);
  std::vector<InitFactor> fac;
  std::vector<InitTerm> terms;
  std::vector<InitItem> items;
  std::vector<double> cvals;  // the CPTs regrouped clique by clique
  cvals.reserve(values.size());
  for (int c = 0; c < nc; ++c) {
    const auto& pv = p.pvars[c];
    std::vector<int64_t> pst(pv.size());
    int64_t sacc = 1;
    for (int i = (int)pv.size() - 1; i >= 0; --i) {
      pst[i] = sacc;
      sacc *= p.card[pv[i]];
    }
    const int64_t cv0 = (int64_t)cvals.size();
    for (int i : by_clique[c]) {
      const int32_t a = cp->fam_off[i], b = cp->fam_off[i + 1];
      fac.push_back(InitFactor{(int64_t)cvals.size() - cv0, (int32_t)terms.size(), b - a});
      cvals.insert(cvals.end(), values.begin() + val_off[i], values.begin() + val_off[i + 1]);
      int64_t fst = 1;
      std::vector<InitTerm> tt(b - a);
      for (int32_t j = b - 1; j >= a; --j) {
        const int32_t v = cp->fam_vars[j];
        const int64_t ps = pst[position(c, v)];
        tt[j - a] = InitTerm{make_udiv((uint32_t)ps), make_udiv((uint32_t)p.card[v]),
                             p.pow2[c] ? log2_exact(ps) : 0, p.card[v], (int32_t)fst, 0};
        fst *= p.card[v];
      }
      terms.insert(terms.end(), tt.begin(), tt.end());
    }
    const int64_t nvals = (int64_t)cvals.size() - cv0;
    cl[c] = InitClique{p.base_off[c], cv0, (int32_t)p.n_entries[c], (int32_t)(fac.size() - by_clique[c].size()),
                       (int32_t)by_clique[c].size(), (int32_t)p.pow2[c],
                       (int32_t)std::min<int64_t>(nvals, INT32_MAX), 0};
    for (int64_t e0 = 0; e0 < p.n_entries[c]; e0 += kInitChunk) items.push_back(InitItem{c, (int32_t)e0});
  }
  cudaStream_t s = (cudaStream_t)stream;
  // the tables may still be read by earlier work on the tree's last stream,
  // or by an allocation-free read-out on a stream of its own
  CU(cudaStreamSynchronize(t->last_stream), "synchronising the tree's last stream");
  if (t->readout_pending) {
    CU(cudaEventSynchronize(t->readout_done), "waiting for a read-out");
    t->readout_pending = false;
  }
  st = t->compute == JT_F64 ? init_typed<double>(t, items, cl, fac, terms, cvals, s, kernel_ms)
                            : init_typed<float>(t, items, cl, fac, terms, cvals, s, kernel_ms);
  if (st != JT_OK) return st;
  std::fill(t->ready.begin(), t->ready.end(), 0);
  return JT_OK;
}

jt_status jt_get_potential(jt_tree t, int32_t clique, double* out) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  const Plan& p = t->plan;
  if (clique < 0 || clique >= p.n_cliques || !out) return fail(JT_ERR_INVALID_ARG, "bad clique or output");
  const CliqueOut co = clique_out(p, clique);
  cudaStream_t strm = t->last_stream;
  cudaError_t e = t->compute == JT_F64
                      ? launch_table_unpermute<double>((const double*)t->base + p.base_off[clique], co,
                                                       t->d_scratch, strm)
                      : launch_table_unpermute<float>((const float*)t->base + p.base_off[clique], co,
                                                      t->d_scratch, strm);
  if (e != cudaSuccess) return cuda_fail(e, "table read-out");
  CU(cudaMemcpyAsync(out, t->d_scratch, (size_t)co.n * sizeof(double), cudaMemcpyDeviceToHost, strm), "table read");
  CU(cudaStreamSynchronize(strm), "table read");
  return JT_OK;
}

jt_status jt_get_info(jt_tree t, jt_tree_info* out) {
  if (!t || !out) return fail(JT_ERR_INVALID_ARG, "null argument");
  out->n_vars = t->plan.n_vars;
  out->n_cliques = t->plan.n_cliques;
  out->depth = t->plan.max_depth;
  out->entries = t->plan.entries;
  out->work_per_case = t->plan.work_per_case;
  out->marginal_len = t->plan.marg_total;
  out->device_bytes = t->device_bytes;
  {
    const Plan& p = t->plan;
    int64_t cb = p.msg_stride * (int64_t)t->elem + 2ll * p.n_cliques * 8 + 4 + (int64_t)p.marg_total * 8 + 8 +
                 (int64_t)p.n_vars * 2 + 2ll * p.n_cliques * 4;
    if (t->flags & JT_MATERIALIZE_CLIQUES) cb += p.base_len * (int64_t)t->elem;
    out->case_bytes = cb;
  }
  out->max_cases = t->max_cases;
  out->compute = t->compute;
  out->flags = t->flags;
  return JT_OK;
}

void jt_free(jt_tree t) { destroy(t); }


jt_status jt_propagate_per_message(jt_tree t, int32_t case_id, int32_t layout, void* stream, float* kernel_ms) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  const Plan& p = t->plan;
  if (case_id < 0 || case_id >= t->max_cases) return fail(JT_ERR_INVALID_ARG, "bad case");
  if (layout != 0 && layout != 1) return fail(JT_ERR_INVALID_ARG, "layout is 0 (naive) or 1 (interleaved)");
  if (!(t->flags & JT_MATERIALIZE_CLIQUES))
    return fail(JT_ERR_STATE, "the per-message propagation works in the calibrated tables: load with "
                              "JT_MATERIALIZE_CLIQUES");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = order_on(t, s)) != JT_OK) return st;
  if ((st = upload_dirty(t, case_id, 1, s)) != JT_OK) return st;
  if (!t->permsg || t->permsg->layout != layout) {
    CU(cudaStreamSynchronize(s), "per-message setup");
    if ((st = build_permsg(t, layout)) != JT_OK) return st;
  }
  // the case's evidence, per clique (stride, cardinality, state)
  std::vector<int16_t> ev((size_t)p.n_vars);
  CU(cudaMemcpyAsync(ev.data(), t->d_ev + (int64_t)case_id * p.n_vars, (size_t)p.n_vars * sizeof(int16_t),
                     cudaMemcpyDeviceToHost, s),
     "evidence read");
  CU(cudaStreamSynchronize(s), "evidence read");
  std::vector<int4> obs;
  std::vector<int> obs_off(1, 0);
  for (int c = 0; c < p.n_cliques; ++c) {
    const auto& pv = p.pvars[c];
    int64_t stv = 1;
    for (int i = (int)pv.size() - 1; i >= 0; --i) {
      const int v = pv[i], e = ev[(size_t)v];
      if (e >= p.card[v]) return fail(JT_ERR_INVALID_ARG, "evidence state out of range");
      if (e >= 0) obs.push_back(make_int4((int)stv, p.card[v], e, 0));
      stv *= p.card[v];
    }
    obs_off.push_back((int)obs.size());
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(cudaEventCreate(&e0), "event");
  CU(cudaEventCreate(&e1), "event");
  cudaError_t err = cudaEventRecord(e0, s);
  if (err == cudaSuccess)
    err = t->compute == JT_F64 ? run_permsg<double>(t, case_id, obs, obs_off, s)
                               : run_permsg<float>(t, case_id, obs, obs_off, s);
  if (err == cudaSuccess) err = cudaEventRecord(e1, s);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_fail(err, "per-message propagation");
  if (kernel_ms) *kernel_ms = ms;
  t->ready[case_id] = 1;
  t->last_stream = s;
  return JT_OK;
}

}  // extern "C"

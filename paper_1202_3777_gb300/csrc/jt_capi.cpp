// C ABI of libjt: tree lifetime, evidence, propagation schedule (CUDA graphs
// of level launches), and read-out.  See include/jt.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "jt_internal.h"
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

constexpr int kCbMax = 8;
constexpr int kMinStages = 3, kMaxStages = 6;   // bulk-copy ring depth (chunks of 16 KB)
constexpr int kRowMax = 4096;                   // rows of one slice held in shared memory
constexpr int kChunkVecs = 2 * kLevelThreads;   // 16-byte vectors per bulk-copy chunk
constexpr int kTwoPerSm = 112 * 1024;           // dynamic shared memory that leaves room for two CTAs
constexpr int kWinMax = 4096;     // max parent-separator entries one collect CTA accumulates
constexpr int kStatusZero = 1, kStatusBadState = 2;

// The schedule of one case range: shared-memory plan, work items, grid.
struct Schedule {
  SmemPlan sp{};
  int32_t grid = 0;
  int32_t n_items = 0;
  DevWork* items = nullptr;       // device
  DevClique* cliques = nullptr;   // device: the tree's descriptors with this schedule's residency
};

struct GraphEntry {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> dev_bufs;    // work lists owned by this graph
  Schedule sched;
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
  void* base = nullptr;
  DevClique* d_cl = nullptr;
  DevPos* d_pos = nullptr;
  DevChild* d_ch = nullptr;
  DevHome* d_hm = nullptr;
  DevSrc* d_src = nullptr;
  DevSrc* d_jh = nullptr;
  int32_t* d_cnt = nullptr;
  VarSrc* d_vs = nullptr;
  int32_t* d_done = nullptr;      // [2][n_cliques][max_cases] dependency flags + the work-queue counter
  int32_t* d_parent = nullptr;
  int32_t* d_err = nullptr;       // set by a kernel whose bounded wait gave up
  DevField* d_fld = nullptr;
  int32_t* d_card = nullptr;
  int32_t* d_moff = nullptr;
  int16_t* d_ev = nullptr;
  void* d_acc = nullptr;
  int64_t acc_stride = 0;
  double* d_ls = nullptr;
  int32_t* d_status = nullptr;
  double* d_marg = nullptr;
  double* d_logz = nullptr;
  void* d_calib = nullptr;
  double* d_scratch = nullptr;    // read-out scratch (sum + clique table)
  int64_t scratch_len = 0;
  int64_t device_bytes = 0;
  // host state
  int16_t* h_ev = nullptr;        // pinned mirror [max_cases][n_vars]
  std::vector<uint8_t> dirty;     // host mirror row newer than the device row
  std::vector<uint8_t> ready;     // a propagation covered the case since its evidence changed
  cudaEvent_t upload_done = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t last_stream = nullptr;
  std::map<std::pair<int, int>, GraphEntry> graphs;
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
    for (void* p : kv.second.dev_bufs) cudaFree(p);
  }
  t->graphs.clear();
}

void destroy(jt_tree t) {
  if (!t) return;
  cudaSetDevice(t->device);
  cudaDeviceSynchronize();
  free_graphs(t);
  void* ptrs[] = {t->base, t->d_cl, t->d_pos, t->d_ch, t->d_hm, t->d_src, t->d_jh, t->d_cnt, t->d_vs, t->d_done, t->d_parent, t->d_err, t->d_fld, t->d_card, t->d_moff,
                  t->d_ev, t->d_acc, t->d_ls, t->d_status, t->d_marg, t->d_logz, t->d_calib, t->d_scratch};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (t->h_ev) cudaFreeHost(t->h_ev);
  if (t->upload_done) cudaEventDestroy(t->upload_done);
  if (t->cap_stream) cudaStreamDestroy(t->cap_stream);
  delete t;
}

// ---------------------------------------------------------------------------
// Schedule for a case range: per level, the CTA slices and shared-memory plan.
// ---------------------------------------------------------------------------

// Work items and the (uniform) shared-memory plan of one propagation over
// n_cases cases: every clique table is cut into slices (multiples of the
// bulk-copy chunk, at most `rowcap` rows, a collect window of at most kWinMax
// parent-separator entries, about two slices per SM per level); cases are
// grouped into blocks of cb.  Shared-memory residency, most valuable first:
// per-slice row sums / row factors and the column joint (touched per entry),
// then factors and outputs (touched per row), which otherwise stay in global
// memory.
jt_status plan_schedule(jt_tree t, int n_cases, Schedule* S, std::vector<DevWork>* items,
                        std::vector<DevClique>* cliques) {
  const Plan& p = t->plan;
  const int VEC = (int)(16 / t->elem);
  const int chunk = kChunkVecs * VEC;       // two vectors per consumer thread per chunk
  int n_child = 0, n_field = 0, n_home = 0, k = 0, facm = 0, rho = 0, outd = 0, jnt = 0;
  for (int c = 0; c < p.n_cliques; ++c) {
    const DevClique& dc = p.dcl[c];
    n_child = std::max(n_child, dc.n_child);
    n_field = std::max(n_field, dc.n_field);
    n_home = std::max(n_home, dc.n_home);
    k = std::max(k, dc.k);
    facm = std::max(facm, p.fac_collect[c]);
    if (c != 0) rho = std::max(rho, dc.sep_size);
    outd = std::max(outd, p.out_dist[c]);
    if (dc.joint_off >= 0) jnt = std::max(jnt, dc.P);
  }
  const int budget = t->smem_max;
  std::vector<int64_t> ctile(p.n_cliques);
  int win = 1, rowmax = 1, cb = 1;
  auto make_tiles = [&](int cbv, int rowcap) {
    win = 1;
    rowmax = 1;
    const int nb = (n_cases + cbv - 1) / cbv;
    for (int d = 0; d <= p.max_depth; ++d) {
      int64_t E = 0;
      for (int c : p.levels[d]) E += p.dcl[c].n;
      const int64_t tiles_wanted = std::max<int64_t>(1, (2ll * t->n_sm) / std::max(1, nb));
      int64_t tile = (E + tiles_wanted - 1) / tiles_wanted;
      tile = std::max<int64_t>(tile, chunk);
      tile = std::min<int64_t>(tile, 1 << 20);
      for (int c : p.levels[d]) {
        const DevClique& dc = p.dcl[c];
        const int64_t L = (int64_t)dc.LR * dc.P;
        // short rows are processed inline while streaming (no per-row buffers)
        const bool inl = inline_rows(dc, VEC);
        int64_t tc = std::min<int64_t>(tile, (int64_t)(kWinMax - 2) * L);
        if (!inl) tc = std::min<int64_t>(tc, (int64_t)(rowcap - 2) * dc.P);
        tc = std::max<int64_t>(chunk, tc / chunk * chunk);
        ctile[c] = tc;
        const int64_t wn = std::min<int64_t>(tc, dc.n) / L + 2;
        win = (int)std::max<int64_t>(win, std::min<int64_t>(wn, dc.sep_size));
        if (!inl) rowmax = (int)std::max<int64_t>(rowmax, std::min<int64_t>(tc, dc.n) / dc.P + 2);
      }
    }
  };
  // fixed part of the layout; what is left of the shared memory becomes the
  // per-case table region, packed clique by clique
  int maxneed = 0;
  for (int c = 0; c < p.n_cliques; ++c) {
    const DevClique& dc = p.dcl[c];
    const int need = p.fac_collect[c] + (c ? dc.sep_size : 0) + p.out_dist[c] + (dc.joint_off >= 0 ? dc.P : 0);
    maxneed = std::max(maxneed, need);
  }
  auto plan_of = [&](int stages, int tabs) {
    return SmemPlan{cb, n_child, n_field, n_home, k, tabs, win, (int32_t)t->elem, stages, chunk, rowmax, 0};
  };
  bool ok = false;
  int tabs = 0;
  for (int cbv = std::min(kCbMax, std::max(1, n_cases)); cbv >= 1 && !ok; cbv = cbv > 1 ? cbv / 2 : 0) {
    cb = cbv;
    for (int rowcap = kRowMax; rowcap >= 64 && !ok; rowcap /= 2) {
      make_tiles(cbv, rowcap);
      const int fixed = SmemLayout(plan_of(kMinStages, 0)).bytes;
      if (fixed > budget) continue;
      const int cap = fixed <= kTwoPerSm ? kTwoPerSm : budget;
      tabs = std::max(0, (cap - fixed - 64) / (cb * (int)t->elem));
      tabs = std::min(tabs, maxneed);
      ok = true;
    }
  }
  if (!ok) return fail(JT_ERR_UNSUPPORTED, "the tree's per-clique tables do not fit in shared memory");
  // deepen the bulk-copy ring with what is left while two CTAs still fit on an SM
  SmemPlan sp = plan_of(kMinStages, tabs);
  const int cap = std::max(SmemLayout(sp).bytes, std::min(budget, kTwoPerSm));
  while (sp.stages < kMaxStages) {
    SmemPlan q = sp;
    q.stages++;
    if (SmemLayout(q).bytes > cap) break;
    sp = q;
  }
  // per-clique residency in the table region: child factors, parent ratio,
  // accumulators, column joint -- in that order while they fit
  cliques->assign(p.dcl.begin(), p.dcl.end());
  for (int c = 0; c < p.n_cliques; ++c) {
    DevClique& dc = (*cliques)[c];
    int off = 0;
    auto place = [&](int n) {
      if (n <= 0 || off + n > tabs) return -1;
      const int o = off;
      off += n;
      return o;
    };
    dc.sm_fac = dc.n_child ? place(p.fac_collect[c]) : -1;
    dc.sm_rho = c ? place(dc.sep_size) : -1;
    dc.sm_out_len = p.out_dist[c];
    dc.sm_out = place(p.out_dist[c]);
    dc.sm_jnt = dc.joint_off >= 0 ? place(dc.P) : -1;
  }
  const int nb = (n_cases + cb - 1) / cb;
  items->clear();
  auto add_level = [&](int d, int collect) {
    for (int c : p.levels[d]) {
      const DevClique& dc = p.dcl[c];
      const int nt = (int)((dc.n + ctile[c] - 1) / ctile[c]);
      for (int ti = 0; ti < nt; ++ti)
        for (int b = 0; b < nb; ++b) {
          DevWork wk{};
          wk.base_off = dc.base_off;
          wk.clique = c;
          wk.t0 = (int32_t)(ti * ctile[c]);
          wk.t1 = (int32_t)std::min<int64_t>(dc.n, (ti + 1) * ctile[c]);
          wk.ntiles = nt;
          wk.cbk = b;
          wk.collect = collect;
          items->push_back(wk);
        }
    }
  };
  for (int d = p.max_depth; d >= 0; --d) add_level(d, 1);  // collect: deepest level first
  for (int d = 0; d <= p.max_depth; ++d) add_level(d, 0);  // distribute: root first
  const int occ = std::max(1, propagate_occupancy((int)t->elem, cb, SmemLayout(sp).bytes));
  if (const char* dbg = std::getenv("JT_DEBUG_PLAN"); dbg && *dbg == '1') {
    int nf = 0, nr = 0, no = 0, nj = 0;
    for (const DevClique& dc : *cliques) {
      nf += dc.sm_fac >= 0;
      nr += dc.sm_rho >= 0;
      no += dc.sm_out >= 0;
      nj += dc.sm_jnt >= 0;
    }
    std::fprintf(stderr,
                 "[jt plan] cases=%d cb=%d items=%zu grid=%d occ=%d smem=%d stages=%d chunk=%d rowmax=%d win=%d "
                 "tabs=%d resident fac/rho/out/jnt=%d/%d/%d/%d of %d cliques\n",
                 n_cases, cb, items->size(), (int)std::min<int64_t>((int64_t)items->size(), (int64_t)t->n_sm * occ), occ,
                 SmemLayout(sp).bytes, sp.stages, sp.chunk, sp.rowmax, sp.win, sp.tabs, nf, nr, no, nj,
                 p.n_cliques);
  }
  S->sp = sp;
  S->n_items = (int32_t)items->size();
  S->grid = (int32_t)std::min<int64_t>(S->n_items, (int64_t)t->n_sm * occ);
  return JT_OK;
}

template <typename T>
LevelArgs<T> level_args(jt_tree t, int case0, int n_cases) {
  LevelArgs<T> a{};
  a.cl = t->d_cl;
  a.pos = t->d_pos;
  a.ch = t->d_ch;
  a.hm = t->d_hm;
  a.src = t->d_src;
  a.jh = t->d_jh;
  a.fld = t->d_fld;
  a.base = (const T*)t->base;
  a.case0 = case0;
  a.n_cases = n_cases;
  a.ev = t->d_ev;
  a.n_vars = t->plan.n_vars;
  a.acc = (T*)t->d_acc;
  a.acc_stride = t->acc_stride;
  a.msg_total = t->plan.msg_total;
  a.marg_total = t->plan.marg_total;
  a.joint_total = t->plan.joint_total;
  a.ls = t->d_ls;
  a.n_cliques = t->plan.n_cliques;
  a.status = t->d_status;
  a.cnt = t->d_cnt;
  a.done = t->d_done;
  a.queue = t->d_done + 2ll * t->plan.n_cliques * t->max_cases;
  a.parent_of = t->d_parent;
  a.err = t->d_err;
  a.max_cases = t->max_cases;
  a.calib = (T*)t->d_calib;
  a.calib_stride = t->plan.base_len;
  return a;
}

// Launch the whole propagation for a case range on `s`: zero the per-case
// accumulators, dependency flags and the work queue, run the persistent
// propagation kernel, finalise.  With `ev` non-null an event is recorded
// before the propagation kernel, between it and the finalisation, and after.
template <typename T>
cudaError_t enqueue_schedule(jt_tree t, int case0, int n_cases, const Schedule& sc, cudaStream_t s,
                             cudaEvent_t* ev) {
  const Plan& p = t->plan;
  cudaError_t err = cudaSuccess;
  auto chk = [&](cudaError_t e) {
    if (err == cudaSuccess && e != cudaSuccess) err = e;
  };
  chk(cudaMemsetAsync((T*)t->d_acc + (int64_t)case0 * t->acc_stride, 0,
                      (size_t)n_cases * t->acc_stride * sizeof(T), s));
  chk(cudaMemsetAsync(t->d_status + case0, 0, (size_t)n_cases * sizeof(int32_t), s));
  chk(cudaMemsetAsync(t->d_done, 0, (2ull * p.n_cliques * t->max_cases + 1) * sizeof(int32_t), s));
  chk(cudaMemsetAsync(t->d_cnt, 0, 2ull * p.n_cliques * t->max_cases * sizeof(int32_t), s));
  LevelArgs<T> a = level_args<T>(t, case0, n_cases);
  a.cl = sc.cliques;
  a.work = sc.items;
  a.n_items = sc.n_items;
  a.cb = sc.sp.cb;
  if (ev) chk(cudaEventRecord(ev[0], s));
  chk(launch_propagate<T>(a, sc.sp, sc.grid, s));
  if (ev) chk(cudaEventRecord(ev[1], s));
  FinalArgs<T> f{};
  f.vs = t->d_vs;
  f.n_vars = p.n_vars;
  f.n_cliques = p.n_cliques;
  f.case0 = case0;
  f.n_cases = n_cases;
  f.acc = (const T*)t->d_acc;
  f.acc_stride = t->acc_stride;
  f.msg_total = p.msg_total;
  f.marg_total = p.marg_total;
  f.ls = t->d_ls;
  f.status = t->d_status;
  f.marg_out = t->d_marg;
  f.logz_out = t->d_logz;
  chk(launch_finalize<T>(f, s));
  if (ev) chk(cudaEventRecord(ev[2], s));
  return err;
}

// Plan the schedule of a case range (work items on the device) and record it
// into a CUDA graph.
template <typename T>
jt_status record_schedule(jt_tree t, int case0, int n_cases, cudaStream_t s, GraphEntry* ge) {
  std::vector<DevWork> items;
  std::vector<DevClique> cliques;
  jt_status st = plan_schedule(t, n_cases, &ge->sched, &items, &cliques);
  if (st != JT_OK) return st;
  DevClique* dcl = nullptr;
  CU(cudaMalloc((void**)&dcl, cliques.size() * sizeof(DevClique)), "clique descriptors");
  ge->dev_bufs.push_back(dcl);
  CU(cudaMemcpy(dcl, cliques.data(), cliques.size() * sizeof(DevClique), cudaMemcpyHostToDevice),
     "clique descriptors");
  ge->sched.cliques = dcl;
  DevWork* dw = nullptr;
  const size_t bytes = std::max<size_t>(1, items.size()) * sizeof(DevWork);
  CU(cudaMalloc((void**)&dw, bytes), "work list");
  ge->dev_bufs.push_back(dw);
  CU(cudaMemcpy(dw, items.data(), items.size() * sizeof(DevWork), cudaMemcpyHostToDevice), "work list upload");
  ge->sched.items = dw;
  CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t err = enqueue_schedule<T>(t, case0, n_cases, ge->sched, s, nullptr);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &g);
  if (err != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(err, "recording the propagation");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
  ge->graph = g;
  CU(cudaGraphInstantiate(&ge->exec, g, 0), "graph instantiate");
  return JT_OK;
}

jt_status get_graph(jt_tree t, int first, int n, GraphEntry** out) {
  auto key = std::make_pair(first, n);
  auto it = t->graphs.find(key);
  if (it == t->graphs.end()) {
    if (t->graphs.size() >= 64) {
      CU(cudaDeviceSynchronize(), "graph cache eviction");
      free_graphs(t);
    }
    GraphEntry ge;
    jt_status st = t->compute == JT_F64 ? record_schedule<double>(t, first, n, t->cap_stream, &ge)
                                        : record_schedule<float>(t, first, n, t->cap_stream, &ge);
    if (st != JT_OK) {
      if (ge.exec) cudaGraphExecDestroy(ge.exec);
      if (ge.graph) cudaGraphDestroy(ge.graph);
      for (void* p : ge.dev_bufs) cudaFree(p);
      return st;
    }
    it = t->graphs.emplace(key, std::move(ge)).first;
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
  t->acc_stride = ((int64_t)3 * p.msg_total + p.marg_total + p.joint_total + 31) / 32 * 32;
  if ((st = alloc(t, (T**)&t->d_acc, t->acc_stride * t->max_cases, "per-case messages")) != JT_OK) return st;
  if (t->flags & JT_MATERIALIZE_CLIQUES) {
    if ((st = alloc(t, (T**)&t->d_calib, p.base_len * t->max_cases, "calibrated tables")) != JT_OK) return st;
  }
  CU(cudaStreamSynchronize(s), "table upload");
  return JT_OK;
}

template <typename V>
jt_status upload_vec(jt_tree t, V** dst, const std::vector<V>& src, const char* what) {
  jt_status st = alloc(t, dst, (int64_t)src.size(), what);
  if (st != JT_OK) return st;
  if (!src.empty()) CU(cudaMemcpy(*dst, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice), what);
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
  int dev = 0;
  CU(cudaGetDevice(&dev), "cudaGetDevice");
  t->device = dev;
  CU(cudaDeviceGetAttribute(&t->n_sm, cudaDevAttrMultiProcessorCount, dev), "device query");
  t->smem_max = smem_budget(dev) - 1024;
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
  if ((st = upload_vec(raw, &raw->d_cl, p.dcl, "descriptors")) != JT_OK) return bail(st);
  if ((st = upload_vec(raw, &raw->d_pos, p.dpos, "descriptors")) != JT_OK) return bail(st);
  if ((st = upload_vec(raw, &raw->d_ch, p.dch, "descriptors")) != JT_OK) return bail(st);
  if ((st = upload_vec(raw, &raw->d_hm, p.dhm, "descriptors")) != JT_OK) return bail(st);
  if ((st = upload_vec(raw, &raw->d_src, p.dsrc, "descriptors")) != JT_OK) return bail(st);
  if ((st = upload_vec(raw, &raw->d_jh, p.djh, "descriptors")) != JT_OK) return bail(st);
  if ((st = upload_vec(raw, &raw->d_vs, p.vsrc, "descriptors")) != JT_OK) return bail(st);
  if ((st = alloc(raw, &raw->d_err, 1, "error word")) != JT_OK) return bail(st);
  if ((st = alloc(raw, &raw->d_done, 2ll * p.n_cliques * raw->max_cases + 1, "dependency flags")) != JT_OK)
    return bail(st);
  if ((st = upload_vec(raw, &raw->d_parent, p.parent, "descriptors")) != JT_OK) return bail(st);
  if (cudaMemset(raw->d_err, 0, sizeof(int32_t)) != cudaSuccess) return bail(fail(JT_ERR_CUDA, "memset"));
  {
    const int64_t ncnt = 2ll * p.n_cliques * raw->max_cases;
    if ((st = alloc(raw, &raw->d_cnt, ncnt, "tile counters")) != JT_OK) return bail(st);
    if (cudaMemset(raw->d_cnt, 0, ncnt * sizeof(int32_t)) != cudaSuccess) return bail(fail(JT_ERR_CUDA, "memset"));
  }
  if ((st = upload_vec(raw, &raw->d_fld, p.dfld, "descriptors")) != JT_OK) return bail(st);
  if ((st = upload_vec(raw, &raw->d_card, p.card, "descriptors")) != JT_OK) return bail(st);
  if ((st = upload_vec(raw, &raw->d_moff, p.moff, "descriptors")) != JT_OK) return bail(st);
  const int64_t nev = (int64_t)raw->max_cases * p.n_vars;
  if ((st = alloc(raw, &raw->d_ev, nev, "evidence")) != JT_OK) return bail(st);
  if (cudaMemset(raw->d_ev, 0xFF, nev * sizeof(int16_t)) != cudaSuccess) return bail(fail(JT_ERR_CUDA, "memset"));
  if ((st = alloc(raw, &raw->d_ls, (int64_t)raw->max_cases * p.n_cliques, "log scales")) != JT_OK) return bail(st);
  if (cudaMemset(raw->d_ls, 0, (size_t)raw->max_cases * p.n_cliques * sizeof(double)) != cudaSuccess)
    return bail(fail(JT_ERR_CUDA, "memset"));
  if ((st = alloc(raw, &raw->d_status, raw->max_cases, "status")) != JT_OK) return bail(st);
  if ((st = alloc(raw, &raw->d_marg, (int64_t)raw->max_cases * p.marg_total, "marginals")) != JT_OK) return bail(st);
  if ((st = alloc(raw, &raw->d_logz, raw->max_cases, "log evidence")) != JT_OK) return bail(st);
  int64_t maxn = 0;
  for (int64_t n : p.n_entries) maxn = std::max(maxn, n);
  raw->scratch_len = maxn + 2;
  if ((st = alloc(raw, &raw->d_scratch, raw->scratch_len, "read-out scratch")) != JT_OK) return bail(st);
  cudaError_t e = cudaMallocHost((void**)&raw->h_ev, (size_t)nev * sizeof(int16_t));
  if (e != cudaSuccess) return bail(cuda_fail(e, "pinned evidence mirror"));
  std::fill(raw->h_ev, raw->h_ev + nev, (int16_t)-1);
  raw->dirty.assign(raw->max_cases, 0);
  raw->ready.assign(raw->max_cases, 0);
  if ((e = cudaEventCreateWithFlags(&raw->upload_done, cudaEventDisableTiming)) != cudaSuccess)
    return bail(cuda_fail(e, "event"));
  if ((e = cudaEventRecord(raw->upload_done, s)) != cudaSuccess) return bail(cuda_fail(e, "event"));
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
  if ((st = upload_dirty(t, first, n, s)) != JT_OK) return st;
  GraphEntry* ge = nullptr;
  if ((st = get_graph(t, first, n, &ge)) != JT_OK) return st;
  CU(cudaGraphLaunch(ge->exec, s), "graph launch");
  for (int i = first; i < first + n; ++i) t->ready[i] = 1;
  t->last_stream = s;
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
  if ((st = upload_dirty(t, first, n, s)) != JT_OK) return st;
  GraphEntry* ge = nullptr;
  if ((st = get_graph(t, first, n, &ge)) != JT_OK) return st;
  std::vector<cudaEvent_t> ev(nl + 1, nullptr);
  for (auto& e : ev) CU(cudaEventCreate(&e), "event");
  cudaError_t err = t->compute == JT_F64 ? enqueue_schedule<double>(t, first, n, ge->sched, s, ev.data())
                                         : enqueue_schedule<float>(t, first, n, ge->sched, s, ev.data());
  if (err == cudaSuccess) err = cudaEventSynchronize(ev[nl]);
  for (int i = 0; i < nl && err == cudaSuccess; ++i) err = cudaEventElapsedTime(&launch_ms[i], ev[i], ev[i + 1]);
  for (auto& e : ev) cudaEventDestroy(e);
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

jt_status jt_get_clique(jt_tree t, int32_t case_id, int32_t clique, double* out) {
  jt_status st = check_tree(t);
  if (st != JT_OK) return st;
  const Plan& p = t->plan;
  if (case_id < 0 || case_id >= t->max_cases || clique < 0 || clique >= p.n_cliques || !out)
    return fail(JT_ERR_INVALID_ARG, "bad case, clique or output");
  if (!(t->flags & JT_MATERIALIZE_CLIQUES)) return fail(JT_ERR_STATE, "tree loaded without JT_MATERIALIZE_CLIQUES");
  if (!t->ready[case_id]) return fail(JT_ERR_STATE, "case not propagated since its evidence changed");
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
  cudaStream_t strm = t->last_stream;
  const int64_t off = (int64_t)case_id * p.base_len + p.base_off[clique];
  cudaError_t e = t->compute == JT_F64
                      ? launch_get_clique<double>((const double*)t->d_calib + off, co, t->d_scratch + 1,
                                                  t->d_scratch, strm)
                      : launch_get_clique<float>((const float*)t->d_calib + off, co, t->d_scratch + 1,
                                                 t->d_scratch, strm);
  if (e != cudaSuccess) return cuda_fail(e, "clique read-out");
  CU(cudaMemcpyAsync(out, t->d_scratch + 1, (size_t)co.n * sizeof(double), cudaMemcpyDeviceToHost, strm),
     "clique read");
  CU(cudaStreamSynchronize(strm), "clique read");
  int32_t code = 0;
  if ((st = case_status(t, case_id, &code)) != JT_OK) return st;
  if (code != JT_OK) return fail((jt_status)code, "case has no posterior");
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
  out->max_cases = t->max_cases;
  out->compute = t->compute;
  out->flags = t->flags;
  return JT_OK;
}

void jt_free(jt_tree t) { destroy(t); }

}  // extern "C"

// Whole-tree propagation of small junction trees: one CTA propagates one
// evidence case at a time, with the case's messages, ratios and stage totals
// in shared memory.
//
// For trees whose per-case state fits one CTA (the 32-clique tree of ternary
// variables, the 1024-clique binary tree, ...) the persistent kernel's
// cross-CTA machinery -- per-block completion counters, bounded polls,
// descriptor blobs fetched per item, messages reduced in L2 -- costs more
// than the work: a propagation is a chain of 2 x depth dependent levels of a
// few thousand entries each.  Here the levels are separated by CTA barriers
// instead.  A level is the set of stages (cliques in one pass) at one depth:
// collect from the deepest level up (Algorithm 2), distribute from the root
// down (Algorithm 3); within a level every stage is independent, and each
// warp takes segments of up to kSmallSeg entries of its stages:
//
//   f(x) = phi_c(x) E(x) prod_g mu_g[key_g(x)] (rho_c[key_p(x)] in the distribute pass)
//   out[key_o(x)] += f(x) for every output port; the stage total += f(x)
//
// with the same quantities as the persistent kernel (Eq. 1-3 with the
// messages scaled to mean one, mu_g = u_g |S_g| / sigma_g, and the ratio
// rho_c = delta_c (sigma_c / Delta_parent) / u_c with 0/0 := 0), so the
// finalisation kernel reads the case's message row and stage totals
// unchanged.  (Finalising in this kernel was measured slower: its FP64 sums
// and divisions then run on one SM, whose FP64 rate on this part is small.)
//
// Latency matters here (a single case of a small tree is a chain of
// 2 x depth levels on one SM): every level's descriptors stay in shared
// memory when they fit, segments are 32 entries so that a level's work
// spreads over every warp, and evidence is tested only on the positions the
// case observes.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "jt_device.cuh"

namespace jt {
namespace {

constexpr int kSmallThreads = 1024;

// Add v at tab[key] for every lane of the warp, where runs of consecutive
// lanes share a key (a key over digits above the lanes' entries): an
// inclusive scan of each run's values (five shuffle steps, restarted at run
// boundaries) leaves the run's sum in its last lane, which issues the one
// shared-memory addition of the run.  Lanes without an entry carry v = 0 and
// a key of their own choosing (their lane's previous key).
template <typename T>
__device__ __forceinline__ void add_runs(T* tab, uint32_t key, T v, int lane) {
  const uint32_t prev = __shfl_up_sync(kFull, key, 1);
  const uint32_t next = __shfl_down_sync(kFull, key, 1);
  const bool head = lane == 0 || prev != key;
  // run start of this lane: the highest head at or below it
  const uint32_t heads = __ballot_sync(kFull, head);
  const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T w = __shfl_up_sync(kFull, v, o);
    if (lane - o >= start) v += w;
  }
  const bool tail = lane == 31 || next != key;
  if (tail && v != T(0)) atomicAdd(tab + key, v);
}

template <typename T, bool POW2>
__device__ __forceinline__ void run_segment(const SmallArgs<T>& a, const T* base, const unsigned char* blob, int e0,
                                            T* msg, const T* rho, const T* scale, const int16_t* ev,
                                            double* sums, int cs, int lane) {
  const DevStage& S = *reinterpret_cast<const DevStage*>(blob);
  const DevPort* port = reinterpret_cast<const DevPort*>(blob + sizeof(DevStage));
  const DevField* fld = reinterpret_cast<const DevField*>(port + S.np);
  const DevPos* pos = reinterpret_cast<const DevPos*>(fld + S.nf);
  const int e1 = min(S.n, e0 + kSmallSeg);
  // the case's observed positions of the stage (bit i = position i), found
  // once per segment; a state beyond the cardinality marks the case and
  // masks nothing
  uint32_t obs = 0u;
  for (int i = lane; i < S.k; i += 32) {
    const int st = ev[pos[i].var];
    if (st < 0) continue;
    if (st >= pos[i].card_ev) atomicOr(&a.status[cs], kStatusBadState);
    else obs |= 1u << i;
  }
  obs = __reduce_or_sync(kFull, obs);
  // (the segment's total in the element type -- at most kSmallSeg terms per
  // lane group -- then once per warp into the stage total in FP64)
  T acc = T(0);
  for (int eb = e0; eb < e1; eb += 32) {   // warp-uniform: every lane takes part in the run sums
    const int e = eb + lane;
    const bool valid = e < e1;
    T f = valid ? base[S.base_off + e] : T(0);
    for (uint32_t m = obs; m != 0u; m &= m - 1u) {
      const DevPos& P = pos[__ffs(m) - 1];
      const uint32_t d = POW2 ? ((uint32_t)e >> P.sh) & ((1u << P.cb) - 1u) : digit_of((uint32_t)e, P);
      if (d != (uint32_t)ev[P.var]) f = T(0);
    }
    if (f != T(0)) {
      for (int pi = 0; pi < S.nin; ++pi) {
        const DevPort& P = port[pi];
        const uint32_t key = key_of<POW2>((uint32_t)e, fld + P.f0, P.nf);
        f *= P.kind == kPortMu ? msg[P.tab + key] * scale[P.other] : rho[P.tab + key];
      }
    }
    for (int pi = S.nin; pi < S.np; ++pi) {
      const DevPort& P = port[pi];
      // (a lane past the segment adds zero at key 0, inside every table)
      const uint32_t key = valid ? key_of<POW2>((uint32_t)e, fld + P.f0, P.nf) : 0u;
      add_runs(msg + P.tab, key, f, lane);
    }
    acc += f;
  }
  acc = warp_sum(acc);
  if (lane == 0 && acc != T(0)) atomicAdd(sums + S.sum_slot, (double)acc);
}

template <typename T>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small(const SmallArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (a.trace != nullptr && blockIdx.x == 0 && threadIdx.x == 0) a.trace[0] = global_ns();
  const int nc = a.n_cliques;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kSmallThreads / 32;
  T* msg = reinterpret_cast<T*>(smem);                                   // [msg_stride]
  T* rho = msg + a.msg_stride;                                           // [msg_total], like the u tables
  double* sums = reinterpret_cast<double*>(smem + (((a.msg_stride + a.msg_total) * sizeof(T) + 15) & ~size_t(15)));
  T* scale = reinterpret_cast<T*>(sums + 2 * nc);                        // [nc] |S_c| / sigma_c
  // (every region from here starts on a 16-byte boundary: the staged
  // descriptors are read as 16-byte units)
  int16_t* ev = reinterpret_cast<int16_t*>(reinterpret_cast<unsigned char*>(sums) + ((3 * nc * 8 + 15) & ~15));
  uint4* lvd = reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(ev) + ((2 * a.n_vars + 15) & ~15));
  // then, when they fit: the clique tables and the packed indices, staged
  // once per CTA (and every level's descriptors, lv_blob_max then covering
  // all of them)
  unsigned char* after = reinterpret_cast<unsigned char*>(lvd + a.lv_blob_max);
  const T* base = a.base;
  if (a.base_in_smem) {
    T* sb = reinterpret_cast<T*>(after);
    const uint4* src = reinterpret_cast<const uint4*>(a.base);
    uint4* dst = reinterpret_cast<uint4*>(sb);
    const int64_t n16 = a.base_len * (int64_t)sizeof(T) / 16;
    for (int64_t i = tid; i < n16; i += kSmallThreads) dst[i] = __ldg(src + i);
    base = sb;
    after += a.base_len * sizeof(T);
  }
  const int32_t* ix = a.idx;
  if (a.idx_in_smem) {
    const uint4* src = reinterpret_cast<const uint4*>(a.idx);
    uint4* dst = reinterpret_cast<uint4*>(after);
    for (int i = tid; i < a.idx_len / 4; i += kSmallThreads) dst[i] = __ldg(src + i);
    ix = reinterpret_cast<const int32_t*>(after);
  }
  if (a.desc_resident) {
    for (int i = tid; i < a.lv_blob_max; i += kSmallThreads) lvd[i] = __ldg(a.blobs + i);
  }
  __syncthreads();
  const int32_t* lv_blob_off = ix;
  const int32_t* seg_lv = ix + a.o_seg_lv;
  const int32_t* lv_stage_off = ix + a.o_lv_stage_off;
  const int32_t* stage_blob = ix + a.o_stage_blob;
  const int32_t* lv_stage = ix + a.o_lv_stage;
  const int32_t* sep_size = ix + a.o_sep_size;
  const int2* segs = reinterpret_cast<const int2*>(ix + a.o_segs);
  if (a.span != nullptr && tid == 0) atomicMin(a.span, (unsigned long long)global_ns());
  // JT_TRACE: CTA 0's first case, [0] kernel start, [1] prologue done, then
  // per level its start and the ends of its first phase (scales and ratios),
  // its segments, and (unused, equal) a third stamp
  uint64_t* tr = (a.trace != nullptr && blockIdx.x == 0) ? a.trace : nullptr;
  if (tr != nullptr && tid == 0) tr[1] = global_ns();
  for (int cs = a.case0 + (int)blockIdx.x; cs < a.case0 + a.n_cases; cs += (int)gridDim.x) {
    if (tid == 0) a.status[cs] = 0;
    for (int64_t i = tid; i < a.msg_stride; i += kSmallThreads) msg[i] = T(0);
    for (int i = tid; i < 2 * nc; i += kSmallThreads) sums[i] = 0.0;
    for (int i = tid; i < nc; i += kSmallThreads) scale[i] = T(0);
    for (int i = tid; i < a.n_vars; i += kSmallThreads) ev[i] = a.ev[(int64_t)cs * a.n_vars + i];
    __syncthreads();
    for (int lv = 0; lv < a.levels; ++lv) {
      if (tr != nullptr && tid == 0) tr[2 + 4 * lv] = global_ns();
      const uint4* lvl = a.desc_resident ? lvd + lv_blob_off[lv] : lvd;   // this level's descriptors
      if (!a.desc_resident) {
        for (int i = lv_blob_off[lv] + tid; i < lv_blob_off[lv + 1]; i += kSmallThreads)
          lvd[i - lv_blob_off[lv]] = __ldg(a.blobs + i);
        __syncthreads();
      }
      // first phase, one barrier: the scales |S_c| / sigma_c of the previous
      // level's collect messages (the totals are complete; this level's
      // parents read them), and the ratios of the own separators of this
      // level's distribute stages (a warp per stage)
      if (lv > 0)
        for (int j = lv_stage_off[lv - 1] + tid; j < lv_stage_off[lv]; j += kSmallThreads) {
          const int st = lv_stage[j];
          if (st >= nc) continue;
          const double sg = sums[st];
          scale[st] = sg > 0.0 ? (T)((double)sep_size[st] / sg) : T(0);
        }
      for (int j = lv_stage_off[lv] + warp; j < lv_stage_off[lv + 1]; j += nw) {
        const int st = lv_stage[j];
        if (st < nc) continue;
        const unsigned char* blob = reinterpret_cast<const unsigned char*>(lvl + stage_blob[st]);
        const DevStage& S = *reinterpret_cast<const DevStage*>(blob);
        const DevPort* port = reinterpret_cast<const DevPort*>(blob + sizeof(DevStage));
        for (int pi = 0; pi < S.nin; ++pi) {
          const DevPort& P = port[pi];
          if (P.kind != kPortRho) continue;
          const double dp = sums[nc + P.other2];
          const T sc = dp > 0.0 ? (T)(sums[P.other] / dp) : T(0);
          for (int k = lane; k < P.size; k += 32) {
            const T u = msg[P.tab + k], d = msg[a.msg_total + P.tab + k];
            rho[P.tab + k] = u > T(0) ? d * sc / u : T(0);
          }
        }
      }
      __syncthreads();
      if (tr != nullptr && tid == 0) tr[3 + 4 * lv] = global_ns();
      for (int sg = seg_lv[lv] + warp; sg < seg_lv[lv + 1]; sg += nw) {
        const int2 g = segs[sg];
        const unsigned char* blob = reinterpret_cast<const unsigned char*>(lvl + stage_blob[g.x]);
        if (reinterpret_cast<const DevStage*>(blob)->bits >= 0)
          run_segment<T, true>(a, base, blob, g.y, msg, rho, scale, ev, sums, cs, lane);
        else
          run_segment<T, false>(a, base, blob, g.y, msg, rho, scale, ev, sums, cs, lane);
      }
      __syncthreads();
      if (tr != nullptr && tid == 0) tr[4 + 4 * lv] = tr[5 + 4 * lv] = global_ns();
    }
    tr = nullptr;
    T* row = a.msg + (int64_t)cs * a.msg_stride;
    for (int64_t i = tid; i < a.msg_stride; i += kSmallThreads) row[i] = msg[i];
    for (int i = tid; i < 2 * nc; i += kSmallThreads) a.sums[(int64_t)cs * 2 * nc + i] = sums[i];
    __syncthreads();
  }
  if (a.span != nullptr && tid == 0) atomicMax(a.span + 1, (unsigned long long)global_ns());
}

std::mutex g_small_mu;

template <typename T>
cudaError_t set_small_attrs() {
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_small_mu);
  if (!done[dev]) {
    e = cudaFuncSetAttribute(k_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_budget(dev, 1));
    if (e != cudaSuccess) return e;
    done[dev] = true;
  }
  return cudaSuccess;
}

}  // namespace

template <typename T>
cudaError_t launch_small(const SmallArgs<T>& a, int grid, int smem, cudaStream_t s) {
  if (grid <= 0 || a.n_cases <= 0) return cudaSuccess;
  cudaError_t e = set_small_attrs<T>();
  if (e != cudaSuccess) return e;
  k_small<T><<<grid, kSmallThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_small<float>(const SmallArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_small<double>(const SmallArgs<double>&, int, int, cudaStream_t);

}  // namespace jt

// Propagation kernels for Hugin belief propagation on sm_103a.
//
// One persistent launch runs a whole propagation (Algorithm 4): collect
// (Algorithm 2) then distribute (Algorithm 3) for a range of evidence cases.
// Work items are blocks of clique tables; every item belongs to a "stage"
// (one clique in one pass) and reads or writes a handful of small tables
// ("ports", see jt_internal.h) through contiguous windows held in shared
// memory:
//
//   collect, clique c (Eq. 2):
//       f(x)  = phi_c(x) E(x) prod_g mu_g[key_g(x)]
//       u_c[key_p(x)] += f(x),   sigma_c += f(x)
//   distribute, clique c (Eq. 3, then Eq. 2 towards every child):
//       f(x)  = phi_c(x) E(x) prod_g mu_g[key_g(x)] rho_c[key_p(x)]
//       delta_g[key_g(x)] += f(x),  joint_c[key_priv(x)] += f(x),  Delta_c += f(x)
//
// mu_g = u_g |S_g| / sigma_g is the child's collect message normalised to
// mean one, rho_c = (delta_c / Delta_parent) / (u_c / sigma_c) the new/old
// ratio of c's own separator with 0/0 := 0, E the evidence indicator.  Each
// stage's total (sigma or Delta) accumulates in FP64; log Z(e) =
// sum_c (log sigma_c - log |S_c|) + log Delta_root.  The root has no collect
// stage: its distribute pass computes the same total.
//
// A CTA has 16 consumer warps and one producer warp.  The producer takes
// items from a global queue (ordered so that every dependency of an item
// comes earlier), hands them to the consumers through a small shared-memory
// FIFO, and streams each block's table into a ring of 16 KB stages with
// cp.async.bulk, running ahead of the consumers across items.  Consumers wait
// (bounded) only for the stages an item reads, i.e. on per-stage counters of
// finished blocks.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "jt_device.cuh"

namespace jt {
namespace {


// Add v at tab[key] for every lane of a full warp; when every lane has the
// same key the warp reduces first and issues one atomic.
template <typename T>
__device__ __forceinline__ void add_combined(uint32_t tab, uint32_t key, T v, int lane) {
  const uint32_t k0 = __shfl_sync(kFull, key, 0);
  if (__all_sync(kFull, key == k0)) {
    v = warp_sum(v);
    if (lane == 0 && v != T(0)) sred_add(tab + k0 * (uint32_t)sizeof(T), v);
  } else if (v != T(0)) {
    sred_add(tab + key * (uint32_t)sizeof(T), v);
  }
}

// Add the entries of a vector (keys ka + dva[j]) summed over the lanes that
// differ from this one only in the bits of `lf` (lanes that share the keys).
// Instead of one butterfly per entry, the first free lane bit halves the
// entries each lane carries, the second halves them again, and the remaining
// bits reduce the one entry left: 6 shuffles and one atomic per lane group
// for four entries and five free bits, where separate butterflies take 20
// shuffles and four atomics.  `ka` is the group's lowest lane's (that lane
// is active whenever any lane of the group is).
__device__ __forceinline__ void scatter_vec(uint32_t ka, const float (&v)[4], uint32_t lf, int lane, bool act,
                                            const int4 dv) {
  if (lf == 0u) {
    if (act) {
      if (v[0] != 0.f) sred_add(ka + (uint32_t)dv.x * 4u, v[0]);
      if (v[1] != 0.f) sred_add(ka + (uint32_t)dv.y * 4u, v[1]);
      if (v[2] != 0.f) sred_add(ka + (uint32_t)dv.z * 4u, v[2]);
      if (v[3] != 0.f) sred_add(ka + (uint32_t)dv.w * 4u, v[3]);
    }
    return;
  }
  const uint32_t m1 = lf & (0u - lf);
  const bool h1 = (lane & m1) != 0u;
  float s0 = h1 ? v[2] : v[0], s1 = h1 ? v[3] : v[1];
  s0 += __shfl_xor_sync(kFull, h1 ? v[0] : v[2], m1);
  s1 += __shfl_xor_sync(kFull, h1 ? v[1] : v[3], m1);
  // this lane now carries entries (0, 1) or (2, 3)
  const int d0 = h1 ? dv.z : dv.x, d1 = h1 ? dv.w : dv.y;
  uint32_t rest = lf & ~m1;
  if (rest == 0u) {
    if (s0 != 0.f) sred_add(ka + (uint32_t)d0 * 4u, s0);
    if (s1 != 0.f) sred_add(ka + (uint32_t)d1 * 4u, s1);
    return;
  }
  const uint32_t m2 = rest & (0u - rest);
  const bool h2 = (lane & m2) != 0u;
  float t = h2 ? s1 : s0;
  t += __shfl_xor_sync(kFull, h2 ? s0 : s1, m2);
  const int dj = h2 ? d1 : d0;
  rest &= ~m2;
#pragma unroll
  for (int b = 1; b < 32; b <<= 1)
    if (rest & (uint32_t)b) t += __shfl_xor_sync(kFull, t, b);
  if ((lane & rest) == 0u && t != 0.f) sred_add(ka + (uint32_t)dj * 4u, t);
}
__device__ __forceinline__ void scatter_vec(uint32_t ka, const double (&v)[2], uint32_t lf, int lane, bool act,
                                            const int4 dv) {
  if (lf == 0u) {
    if (act) {
      if (v[0] != 0.0) sred_add(ka + (uint32_t)dv.x * 8u, v[0]);
      if (v[1] != 0.0) sred_add(ka + (uint32_t)dv.y * 8u, v[1]);
    }
    return;
  }
  const uint32_t m1 = lf & (0u - lf);
  const bool h1 = (lane & m1) != 0u;
  double t = h1 ? v[1] : v[0];
  t += __shfl_xor_sync(kFull, h1 ? v[0] : v[1], m1);
  const uint32_t rest = lf & ~m1;
#pragma unroll
  for (int b = 1; b < 32; b <<= 1)
    if (rest & (uint32_t)b) t += __shfl_xor_sync(kFull, t, b);
  if ((lane & rest) == 0u && t != 0.0) sred_add(ka + (uint32_t)(h1 ? dv.y : dv.x) * 8u, t);
}

// Add, for every case c of a case block, v[c] summed over the lanes that
// differ from this one only in the bits of `rest` at ka + (c0 + c) * wstride
// (one key per lane group; `ka` the group's).  Each free lane bit first
// halves the cases a lane carries (the lane keeps one half, sends the other
// to its partner), so the cases end up spread over the group's lanes and one
// atomic per holding lane adds them: for 8 cases and 4 free bits, 9 shuffles
// instead of 32.
template <typename T, int N>
struct CaseScatter {
  __device__ __forceinline__ static void run(uint32_t ka, uint32_t wstride, const T (&v)[N], uint32_t c0,
                                             uint32_t rest, int lane) {
    if (rest == 0u) {
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (v[i] != T(0)) sred_add(ka + (c0 + (uint32_t)i) * wstride, v[i]);
      return;
    }
    const uint32_t m = rest & (0u - rest);
    const bool h = (lane & m) != 0u;
    T w[N / 2];
#pragma unroll
    for (int i = 0; i < N / 2; ++i)
      w[i] = (h ? v[i + N / 2] : v[i]) + __shfl_xor_sync(kFull, h ? v[i] : v[i + N / 2], m);
    CaseScatter<T, N / 2>::run(ka, wstride, w, c0 + (h ? (uint32_t)(N / 2) : 0u), rest & ~m, lane);
  }
};
template <typename T>
struct CaseScatter<T, 1> {
  __device__ __forceinline__ static void run(uint32_t ka, uint32_t wstride, const T (&v)[1], uint32_t c0,
                                             uint32_t rest, int lane) {
    T t = v[0];
#pragma unroll
    for (int b = 1; b < 32; b <<= 1)
      if (rest & (uint32_t)b) t += __shfl_xor_sync(kFull, t, b);
    if ((lane & rest) == 0u && t != T(0)) sred_add(ka + c0 * wstride, t);
  }
};

// ---- control warp 2: preparation of the next item ---------------------------
// For the item in buffer b: wait for its blob and dependencies, enter the
// evidence (block-level digits into the block factor, in-block digits into
// per-case lists), fold block-constant inputs and child-message scales into
// the block factor, and fill the windows (child messages by bulk copy, own
// separator ratios computed, outputs zeroed).  The item is ready for the
// consumers when pfull[b] completes (including the copies' bytes).
template <typename T, int CB>
__device__ __forceinline__ void prep_lanes(const PropArgs<T>& a, const Smem& s0) {
  constexpr unsigned kMask = kFull;         // the whole preparation warp
  constexpr int NL = 32;
  constexpr int U = 4;                      // tasks per lane per round (their loads in flight together)
  const int pl = (int)(threadIdx.x & 31);
  for (uint32_t slot = 0;; ++slot) {
    const uint32_t b = slot & 1u, par = (slot >> 1) & 1u;
    bool ok = mbar_wait(s0.ifull + b, par, a.err, s0.misc, a.wait_ns);
    ok = __all_sync(kMask, ok);
    if (!ok) break;
    ItemInfo& inf = s0.info[b];
    const DevItem w = inf.w;
    if (w.stage < 0) {  // sentinel: pass it on
      __syncwarp(kMask);
      if (pl == 0) mbar_arrive(s0.pfull + b);
      break;
    }
    ok = __all_sync(kMask, mbar_wait(s0.bfull + b, par, a.err, s0.misc, a.wait_ns));
    if (!ok) break;
    const Smem s = with_buffer(s0, b);
    const DevStage S = *s.stage;
    const int cb0 = a.case0 + w.cbk * CB;
    const int ncb = min(CB, a.case0 + a.n_cases - cb0);
    const uint32_t eb = (uint32_t)w.block * (uint32_t)S.B;
    const bool fast = S.bits >= 0;
    uint64_t* tr = a.trace != nullptr ? a.trace + (int64_t)inf.idx * kTraceSlots : nullptr;
    if (tr != nullptr && pl == 0) tr[11] = global_ns();
    // what needs no other item comes before the dependency wait (off the
    // critical path): the evidence and the zeroed output windows
    if (pl < CB) {
      s.nobs[pl] = 0;
      s.bf[pl] = 1.0;
    }
    __syncwarp(kMask);
    // evidence (block-level digits into the block factor, in-block digits
    // into per-case lists)
    const int nev = ncb * S.k;
    for (int t0 = pl; t0 < nev; t0 += U * NL) {
      int sv[U];
#pragma unroll
      for (int r = 0; r < U; ++r) {
        const int t = t0 + r * NL;
        sv[r] = -1;
        if (t >= nev) continue;
        const int cl = t / S.k, i = t - cl * S.k;
        sv[r] = a.ev[(int64_t)(cb0 + cl) * a.n_vars + s.pos[i].var];
      }
#pragma unroll
      for (int r = 0; r < U; ++r) {
        const int t = t0 + r * NL;
        const int st = sv[r];
        if (t >= nev || st < 0) continue;
        const int cl = t / S.k, i = t - cl * S.k;
        const DevPos& P = s.pos[i];
        if (st >= P.card_ev) {
          atomicOr(&a.status[cb0 + cl], kStatusBadState);
          continue;
        }
        if (fast) {
          const int inside = max(0, min(P.cb, S.bits - P.sh));
          const uint32_t lo_m = (1u << inside) - 1u;
          const uint32_t hi_d = (eb >> P.sh) & ((1u << P.cb) - 1u);
          if (hi_d != ((uint32_t)st & ~lo_m)) {
            s.bf[cl] = 0.0;
          } else if (lo_m != 0u) {
            const int slot2 = atomicAdd(&s.nobs[cl], 1);
            s.obs[cl * a.max_k + slot2] = make_int4(P.sh, (int)lo_m, st & (int)lo_m, i);
          }
        } else if (i < S.k - S.kin) {
          if (digit_of(eb, P) != (uint32_t)st) s.bf[cl] = 0.0;
        } else {
          const int slot2 = atomicAdd(&s.nobs[cl], 1);
          s.obs[cl * a.max_k + slot2] = make_int4(i, 0, st, i);
        }
      }
    }
    {
      // (a window the consumers store whole needs no zeros; 16-byte stores:
      // windows are allocated in whole groups of 4 entries)
      const uint32_t win32 = smem_u32(s.win);
      constexpr int VEC = VecT<T>::N;
      const T z[VEC] = {};
      for (int pi = S.nin; pi < S.np; ++pi) {
        const DevPort& P = s.port[pi];
        if (P.K <= 1 || ((P.vmode & kVmodeStore) && fast)) continue;
        const int kr = (P.K + 3) / 4 * 4;
        for (int cl = 0; cl < ncb; ++cl) {
          const uint32_t dst = win32 + (uint32_t)(cl * a.win_max + P.win) * (uint32_t)sizeof(T);
          for (int ii = pl * VEC; ii < kr; ii += NL * VEC) sst_vec(dst + (uint32_t)ii * (uint32_t)sizeof(T), z);
        }
      }
    }
    // dependencies
    bool dok = true;
    if (S.ndep > 0) dok = await_deps(a.deps + S.dep0, S.ndep, a.done, a.n_cb, w.cbk, a.err, s.misc, pl, NL, kMask, a.wait_ns);
    if (tr != nullptr && pl == 0) tr[10] = global_ns();
    // the child-message windows first (bulk copies; the consumers wait for their bytes)
    uint32_t bulk_bytes = 0;
    if (dok) {
      for (int pi = 0; pi < S.nin; ++pi) {
        const DevPort& P = s.port[pi];
        if (P.K > 1 && P.kind == kPortMu && bulk_window<T>(S, P)) bulk_bytes += (uint32_t)(ncb * P.K) * (uint32_t)sizeof(T);
      }
      if (pl == 0) mbar_expect_tx_only(s.pfull + b, bulk_bytes);
      __syncwarp(kMask);
      if (bulk_bytes > 0) {
        fence_proxy_async_all();  // the messages were written by other CTAs (generic and bulk-reduce writes)
        // copy n (port, case) goes to lane n % NL: the lanes find their ports
        // first, then compute the window keys and issue the copies together
        // (up to kBT rounds; any further copies one lane at a time)
        constexpr int kBT = 4;
        int mp[kBT], mc[kBT];
#pragma unroll
        for (int r = 0; r < kBT; ++r) mp[r] = -1, mc[r] = 0;
        int n = 0;
        for (int pi = 0; pi < S.nin; ++pi) {
          const DevPort& P = s.port[pi];
          if (P.K <= 1 || P.kind != kPortMu || !bulk_window<T>(S, P)) continue;
          for (int cl = 0; cl < ncb; ++cl, ++n) {
            if (n % NL != pl) continue;
            const int r = n / NL;
            if (r < kBT) {
#pragma unroll
              for (int q = 0; q < kBT; ++q)
                if (q == r) mp[q] = pi, mc[q] = cl;
              continue;
            }
            const uint32_t kb = key_of<true>(eb, s.fld + P.f0, P.nf);
            const T* src = a.msg + (int64_t)(cb0 + cl) * a.msg_stride + P.tab + kb;
            bulk_g2s(s.win + (size_t)(cl * a.win_max + P.win) * sizeof(T), src, (uint32_t)P.K * (uint32_t)sizeof(T),
                     s.pfull + b);
          }
        }
#pragma unroll
        for (int r = 0; r < kBT; ++r) {
          if (mp[r] < 0) continue;
          const DevPort& P = s.port[mp[r]];
          const int cl = mc[r];
          const uint32_t kb = key_of<true>(eb, s.fld + P.f0, P.nf);
          const T* src = a.msg + (int64_t)(cb0 + cl) * a.msg_stride + P.tab + kb;
          bulk_g2s(s.win + (size_t)(cl * a.win_max + P.win) * sizeof(T), src, (uint32_t)P.K * (uint32_t)sizeof(T),
                   s.pfull + b);
        }
      }
    }
    __syncwarp(kMask);
    if (dok) {
      // per (case, input port): the child message's scale |S|/sigma, or the
      // value of a block-constant input
      const int ntask = ncb * S.nin;
      for (int t0 = pl; t0 < ntask; t0 += U * NL) {
        double x0[U], x1[U], x2[U], x3[U];
#pragma unroll
        for (int r = 0; r < U; ++r) {
          x0[r] = x1[r] = x2[r] = x3[r] = 0.0;
          const int t = t0 + r * NL;
          if (t >= ntask) continue;
          const int cl = t / S.nin, pi = t - cl * S.nin;
          const DevPort& P = s.port[pi];
          const int cs = cb0 + cl;
          const T* row = a.msg + (int64_t)cs * a.msg_stride;
          const double* sums = a.sums + (int64_t)cs * 2 * a.n_cliques;
          if (P.kind == kPortMu) {
            x0[r] = __ldcg(sums + P.other);
            if (P.K <= 1) {
              const uint32_t key = fast ? key_of<true>(eb, s.fld + P.f0, P.nf) : key_of<false>(eb, s.fld + P.f0, P.nf);
              x1[r] = (double)__ldcg(row + P.tab + key);
            }
          } else if (P.kind == kPortRho && P.K <= 1) {
            const uint32_t key = fast ? key_of<true>(eb, s.fld + P.f0, P.nf) : key_of<false>(eb, s.fld + P.f0, P.nf);
            x0[r] = __ldcg(sums + P.other);
            x1[r] = __ldcg(sums + a.n_cliques + P.other2);
            x2[r] = (double)__ldcg(row + P.tab + key);
            x3[r] = (double)__ldcg(row + a.delta_off + P.tab + key);
          }
        }
#pragma unroll
        for (int r = 0; r < U; ++r) {
          const int t = t0 + r * NL;
          if (t >= ntask) continue;
          const int cl = t / S.nin, pi = t - cl * S.nin;
          const DevPort& P = s.port[pi];
          double v = 1.0;
          if (P.kind == kPortMu) {
            v = x0[r] > 0.0 ? (double)P.size / x0[r] : 0.0;
            if (P.K <= 1) v *= x1[r];
          } else if (P.kind == kPortRho && P.K <= 1) {
            v = (x1[r] > 0.0 && x2[r] > 0.0) ? x3[r] * (x0[r] / x1[r]) / x2[r] : 0.0;
          }
          s.pval[cl * a.max_ports + pi] = v;
        }
      }
      // input windows that are not bulk copies: ratios of the own separator,
      // child messages of unaligned windows
      const uint32_t win32 = smem_u32(s.win);
      for (int pi = 0; pi < S.nin; ++pi) {
        const DevPort& P = s.port[pi];
        if (P.K <= 1) continue;
        if (P.kind == kPortMu && bulk_window<T>(S, P)) continue;
        const uint32_t kb = fast ? key_of<true>(eb, s.fld + P.f0, P.nf) : key_of<false>(eb, s.fld + P.f0, P.nf);
        for (int cl = 0; cl < ncb; ++cl) {
          const int cs = cb0 + cl;
          const uint32_t dst = win32 + (uint32_t)(cl * a.win_max + P.win) * (uint32_t)sizeof(T);
          const T* row = a.msg + (int64_t)cs * a.msg_stride + P.tab + kb;
          T sc = T(0);
          if (P.kind == kPortRho) {
            const double* sums = a.sums + (int64_t)cs * 2 * a.n_cliques;
            const double sgc = __ldcg(sums + P.other), dp = __ldcg(sums + a.n_cliques + P.other2);
            sc = dp > 0.0 ? (T)(sgc / dp) : T(0);
          }
          // per entry in the element type (the messages are stored in it;
          // FP64 issue is scarce on this part)
          for (int i0 = pl; i0 < P.K; i0 += U * NL) {
            T u[U], d[U];
#pragma unroll
            for (int r = 0; r < U; ++r) {
              const int ii = i0 + r * NL;
              u[r] = ii < P.K ? __ldcg(row + ii) : T(0);
              d[r] = (ii < P.K && P.kind == kPortRho) ? __ldcg(row + a.delta_off + ii) : T(0);
            }
#pragma unroll
            for (int r = 0; r < U; ++r) {
              const int ii = i0 + r * NL;
              if (ii >= P.K) continue;
              const T v = P.kind == kPortMu ? u[r] : (u[r] > T(0) ? d[r] * sc / u[r] : T(0));
              sst<T>(dst + (uint32_t)ii * (uint32_t)sizeof(T), v);
            }
          }
        }
      }
    }
    __syncwarp(kMask);
    // block factor per case
    if (dok && pl < ncb) {
      double bfv = s.bf[pl];
      for (int pi = 0; pi < S.nin; ++pi) bfv *= s.pval[pl * a.max_ports + pi];
      s.bf[pl] = bfv;
    }
    if (pl == 0) inf.ok = dok ? 1 : 0;
    __syncwarp(kMask);
    if (tr != nullptr && pl == 0) tr[2] = global_ns();
    if (pl == 0) {
      if (!dok) mbar_expect_tx_only(s.pfull + b, 0u);
      mbar_arrive(s.pfull + b);  // completes once the bulk window bytes have landed
    }
    if (!dok) break;  // the consumers see ok = 0 and stop
  }
}

// ---- control warp 1, lane 0: the signalling lane ---------------------------
// For each finished item: add the output windows into the message arrays
// with bulk reductions (the consumers already added the rest), wait until
// they completed, make them visible GPU-wide, count the block as done, and
// free the item's buffer.
template <typename T, int CB>
__device__ __forceinline__ void signaller(const PropArgs<T>& a, const Smem& s0) {
  for (uint32_t k = 0;; ++k) {
    const uint32_t sl = k % kSig;
    if (!mbar_wait(s0.sfull + sl, (k / kSig) & 1u, a.err, s0.misc, a.wait_ns)) break;
    const int4 g = s0.sig[sl];   // stage, case block, buffer, item index
    mbar_arrive(s0.sempty + sl);
    if (g.x < 0) break;
    // the consumers' window writes (generic proxy) before the bulk reads
    fence_proxy_async();
    const uint32_t b = (uint32_t)g.z;
    const Smem s = with_buffer(s0, b);
    const DevStage& S = *s.stage;
    const DevItem& w = s0.info[b].w;
    bool any = false;
    if constexpr (CB == 1) {
      // the block total (left in the block-factor slot): stage total and
      // block-constant outputs
      const uint32_t eb = (uint32_t)w.block * (uint32_t)S.B;
      const int c0 = a.case0 + g.y * CB;
      const int ncb = min(CB, a.case0 + a.n_cases - c0);
      const bool fast = S.bits >= 0;
      for (int cl = 0; cl < ncb; ++cl) {
        const double t = s.bf[cl];
        if (t == 0.0) continue;
        T* row = a.msg + (int64_t)(c0 + cl) * a.msg_stride;
        for (int pi = S.nin; pi < S.np; ++pi) {
          const DevPort& P = s.port[pi];
          if (P.K > 1) continue;
          const uint32_t key = fast ? key_of<true>(eb, s.fld + P.f0, P.nf) : key_of<false>(eb, s.fld + P.f0, P.nf);
          atomicAdd(row + P.tab + key, (T)t);
        }
        atomicAdd(a.sums + (int64_t)(c0 + cl) * 2 * a.n_cliques + S.sum_slot, t);
      }
    }
    if (S.bits >= 0) {
      const uint32_t eb = (uint32_t)w.block * (uint32_t)S.B;
      const int c0 = a.case0 + g.y * CB;
      const int ncb = min(CB, a.case0 + a.n_cases - c0);
      for (int pi = S.nin; pi < S.np; ++pi) {
        const DevPort& P = s.port[pi];
        if (P.K <= 1 || !bulk_window<T>(S, P)) continue;
        const uint32_t kb = key_of<true>(eb, s.fld + P.f0, P.nf);
        for (int cl = 0; cl < ncb; ++cl) {
          T* dst = a.msg + (int64_t)(c0 + cl) * a.msg_stride + P.tab + kb;
          bulk_reduce_add(dst, s.win + (size_t)(cl * a.win_max + P.win) * sizeof(T),
                          (uint32_t)P.K * (uint32_t)sizeof(T));
          any = true;
        }
      }
    }
    if (any) {
      bulk_commit();
      bulk_wait_all();
      fence_proxy_async_all();
    }
    __threadfence();
    atomicAdd(a.done + (int64_t)g.x * a.n_cb + g.y, 1);
    if (a.trace != nullptr && g.w >= 0) a.trace[(int64_t)g.w * kTraceSlots + 9] = global_ns();
    mbar_arrive(s0.wfree + b);
  }
}

// ---- consumers ------------------------------------------------------------


// Stream the chunks of one item (fast path: power-of-two clique, the block
// starts on a vector boundary, at most kMaxFastPorts ports).  An entry's
// offset in the block splits into disjoint bit sets
//     o = io + tid * VEC + j,   io = m * (consumers * VEC)  (iteration m),
// so every port key is kt[i][tid] (fixed per item) + kiter[i][m] (uniform,
// tabulated per item) + dvec[j].  Per vector: evidence, input gathers, the
// block total, and output scatters reduced over the lanes that share a key;
// the key work is shared by every case of the case block.  Two outputs
// accumulate in registers instead: the first output whose vector entries
// share a key (flushed when its key changes, which happens uniformly across
// the CTA), and, for one case, a joint whose key ignores the chunk bits
// (flushed at the end of the item).
template <typename T, int CB>
__device__ __forceinline__ bool stream_fast(const PropArgs<T>& a, const Smem& s, const DevItem& w, int ncb, int cb0,
                                            int n_in, int n_live, int live_off, int ki_off, int kt_o, bool any_obs,
                                            const T (&bfv)[CB], T (&tot)[CB], RingPos& rp) {
  constexpr int NT = consumers_for(CB);
  constexpr int VEC = VecT<T>::N;
  constexpr int VPT = chunk_bytes_for(CB) / (16 * NT);  // vectors per thread per chunk
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t RS = (uint32_t)a.ring, CH = (uint32_t)a.chunk;
  const uint32_t ring32 = smem_u32(s.ring), win32 = smem_u32(s.win);
  // the live ports and key tables in the blob: kt (16-bit) per thread,
  // kiter per iteration, rows of kMaxIter (past the block: the last entry)
  constexpr bool kBlob = CB == 1;   // tables in the blob (16-bit kt) or computed per item (32-bit kt)
  const uint32_t blob32 = smem_u32(s.stage);
  const uint32_t kt32 = kBlob ? blob32 + (uint32_t)kt_o + 2u * (uint32_t)tid : smem_u32(s.kt) + 4u * (uint32_t)tid;
  const uint32_t ki32 = kBlob ? blob32 + (uint32_t)ki_off : smem_u32(s.kiter);
  auto ktld = [&](int i) -> uint32_t {
    return kBlob ? sld_u16(kt32 + 2u * (uint32_t)(i * NT)) : (uint32_t)sld_s32(kt32 + 4u * (uint32_t)(i * NT));
  };
  const uint32_t wstride = (uint32_t)a.win_max * (uint32_t)sizeof(T);  // bytes between cases' windows
  const LivePort* lp = kBlob ? reinterpret_cast<const LivePort*>(reinterpret_cast<const unsigned char*>(s.stage) + live_off)
                             : reinterpret_cast<const LivePort*>(s.live);
  // (the hot loop reads the live-port table and the evidence lists with
  // explicit shared-memory loads)
  const uint32_t lp32 = kBlob ? blob32 + (uint32_t)live_off : smem_u32(s.live);
  const uint32_t nobs32 = smem_u32(s.nobs), obs32 = smem_u32(s.obs);
  const int nchunks = (int)((w.n + CH - 1) / CH);
  // register-accumulated outputs
  int ra = -1, ja = -1;
  for (int i = n_in; i < n_live; ++i) {
    const int32_t md = sld_s32(lp32 + (uint32_t)i * (uint32_t)sizeof(LivePort));
    if (ra < 0 && (md & 3) == 0) ra = i;
    else if (CB == 1 && ja < 0 && (md & 3) != 0 && !(md & (kModeChunk | kModeStore))) ja = i;
  }
  T racc[CB];
#pragma unroll
  for (int cl = 0; cl < CB; ++cl) racc[cl] = T(0);
  uint32_t rkt = 0, rlf = 0, rcur = 0;
  bool rin = true, jiter = true;
  if (ra >= 0) {
    rkt = (uint32_t)ktld(ra);
    rlf = (uint32_t)(lp[ra].mode >> 3) & 31u;
    rcur = (uint32_t)sld_s32(ki32 + 4u * (uint32_t)(ra * kMaxIter));
    rin = (lp[ra].mode & kModeInChunk) != 0;
  }
  if (ja >= 0) jiter = (lp[ja].mode & kModeIter) != 0;
  T jacc[VPT][VEC];
#pragma unroll
  for (int it = 0; it < VPT; ++it)
#pragma unroll
    for (int j = 0; j < VEC; ++j) jacc[it][j] = T(0);
  bool ok = true;
  uint64_t waited = 0;
  for (int ci = 0; ci < nchunks; ++ci, rp.advance(RS)) {
    const uint32_t st = rp.st;
    const uint64_t tw = (a.trace != nullptr && lane == 0) ? global_ns() : 0;
    // the warp leaves together (its lanes reduce with shuffles below)
    if (!__all_sync(kFull, mbar_wait(s.full + st, rp.ph, a.err, s.misc, a.wait_ns))) {
      ok = false;
      break;
    }
    if (a.trace != nullptr && lane == 0) waited += global_ns() - tw;
    const uint32_t sb = ring32 + st * CH * (uint32_t)sizeof(T);
    const uint32_t cbase = (uint32_t)ci * CH;
    const int nvec = (int)(min((uint32_t)w.n - cbase, CH) / VEC);
    // all of this thread's vectors of the chunk first (their loads overlap)
    T xs[VPT][VEC];
#pragma unroll
    for (int it = 0; it < VPT; ++it) {
      if (it * NT + tid < nvec) {
        sld_vec(sb + (uint32_t)(it * NT + tid) * (VEC * (uint32_t)sizeof(T)), xs[it]);
      } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) xs[it][j] = T(0);
      }
    }
    // every vector of this thread in the chunk at once (VPT of them): their
    // gathers and reductions are independent, so their latencies overlap.
    // Lanes past the chunk's end carry zeros.
    bool act[VPT];
    int mi[VPT];               // iteration index within the block
    uint32_t o0[VPT];
    T f[VPT][CB][VEC];
#pragma unroll
    for (int it = 0; it < VPT; ++it) {
      const int vi = it * NT + tid;
      act[it] = vi < nvec;
      mi[it] = ci * VPT + it;
      o0[it] = cbase + (uint32_t)vi * VEC;
#pragma unroll
      for (int cl = 0; cl < CB; ++cl)
#pragma unroll
        for (int j = 0; j < VEC; ++j) f[it][cl][j] = xs[it][j] * bfv[cl];
    }
    // evidence inside the block: each observation read once for all of the
    // thread's vectors
    if (any_obs) {
#pragma unroll
      for (int cl = 0; cl < CB; ++cl) {
        if (bfv[cl] == T(0)) continue;
        const int no = sld_s32(nobs32 + 4u * (uint32_t)cl);
        for (int e = 0; e < no; ++e) {
          const int4 ob = sld_v4s32(obs32 + 16u * (uint32_t)(cl * a.max_k + e));
#pragma unroll
          for (int it = 0; it < VPT; ++it) {
            const uint32_t d = (o0[it] >> ob.x) & (uint32_t)ob.y;
#pragma unroll
            for (int j = 0; j < VEC; ++j)
              if (d + (((uint32_t)j >> ob.x) & (uint32_t)ob.y) != (uint32_t)ob.z) f[it][cl][j] = T(0);
          }
        }
      }
    }
    // input gathers
    for (int i = 0; i < n_in; ++i) {
      const int32_t md = sld_s32(lp32 + (uint32_t)i * (uint32_t)sizeof(LivePort));
      const uint32_t kti = (uint32_t)ktld(i);
      // (a lane past the block's end reads its port window's first entries,
      // which are always filled: its own key may lie outside the window)
      const uint32_t kwin = (uint32_t)sld_s32(lp32 + (uint32_t)i * (uint32_t)sizeof(LivePort) + 8u);
      if (VPT > 1 && CB == 1 && !(md & kModeInChunk)) {
        // the thread's vectors of this chunk share the key: one gather for
        // all (a vector past the block's end multiplies zeros)
        if (bfv[0] == T(0)) continue;
        uint32_t k = kti;
        if (md & kModeIter) k += (uint32_t)sld_s32(ki32 + 4u * (uint32_t)(i * kMaxIter + mi[0]));
        const uint32_t k0 = win32 + (act[0] ? k : kwin) * (uint32_t)sizeof(T);
        const int vm = md & 3;
        T g[VEC];
        if (vm == 1) {
          sld_vec(k0, g);
        } else if (vm == 0) {
          const T g0 = sld<T>(k0);
#pragma unroll
          for (int j = 0; j < VEC; ++j) g[j] = g0;
        } else {
          const int4 dv = sld_v4s32(lp32 + (uint32_t)i * (uint32_t)sizeof(LivePort) + 16u);
          const int dva[4] = {dv.x, dv.y, dv.z, dv.w};
#pragma unroll
          for (int j = 0; j < VEC; ++j) g[j] = sld<T>(k0 + (uint32_t)dva[j] * (uint32_t)sizeof(T));
        }
#pragma unroll
        for (int it = 0; it < VPT; ++it)
#pragma unroll
          for (int j = 0; j < VEC; ++j) f[it][0][j] *= g[j];
        continue;
      }
      uint32_t ka[VPT];
#pragma unroll
      for (int it = 0; it < VPT; ++it) {
        uint32_t k = kti;
        if (md & kModeIter) k += (uint32_t)sld_s32(ki32 + 4u * (uint32_t)(i * kMaxIter + mi[it]));
        ka[it] = win32 + (act[it] ? k : kwin) * (uint32_t)sizeof(T);
      }
      const int vm = md & 3;
      if (vm == 1) {
#pragma unroll
        for (int it = 0; it < VPT; ++it)
#pragma unroll
          for (int cl = 0; cl < CB; ++cl) {
            if (bfv[cl] != T(0)) {
              T g[VEC];
              sld_vec(ka[it] + (uint32_t)cl * wstride, g);
#pragma unroll
              for (int j = 0; j < VEC; ++j) f[it][cl][j] *= g[j];
            }
          }
      } else if (vm == 0) {
#pragma unroll
        for (int it = 0; it < VPT; ++it)
#pragma unroll
          for (int cl = 0; cl < CB; ++cl) {
            if (bfv[cl] != T(0)) {
              const T g = sld<T>(ka[it] + (uint32_t)cl * wstride);
#pragma unroll
              for (int j = 0; j < VEC; ++j) f[it][cl][j] *= g;
            }
          }
      } else {
        const int4 dv = sld_v4s32(lp32 + (uint32_t)i * (uint32_t)sizeof(LivePort) + 16u);
        const int dva[4] = {dv.x, dv.y, dv.z, dv.w};
#pragma unroll
        for (int it = 0; it < VPT; ++it)
#pragma unroll
          for (int cl = 0; cl < CB; ++cl) {
            if (bfv[cl] != T(0)) {
#pragma unroll
              for (int j = 0; j < VEC; ++j)
                f[it][cl][j] *= sld<T>(ka[it] + (uint32_t)cl * wstride + (uint32_t)dva[j] * (uint32_t)sizeof(T));
            }
          }
      }
    }
    T sum[VPT][CB];
#pragma unroll
    for (int it = 0; it < VPT; ++it)
#pragma unroll
      for (int cl = 0; cl < CB; ++cl) {
        sum[it][cl] = T(0);
#pragma unroll
        for (int j = 0; j < VEC; ++j) sum[it][cl] += f[it][cl][j];
        tot[cl] += sum[it][cl];
      }
    // the register-accumulated output: flush when its key changes (the
    // iterations in order)
    if (VPT > 1 && CB == 1 && ra >= 0 && !rin) {
      // a key shared by the thread's vectors of the chunk: one check
      const uint32_t kc = (uint32_t)sld_s32(ki32 + 4u * (uint32_t)(ra * kMaxIter + mi[0]));
      if (kc != rcur) {
        const uint32_t ra_a = win32 + (rkt + rcur) * (uint32_t)sizeof(T);
        CaseScatter<T, CB>::run(rlf != 0u ? __shfl_sync(kFull, ra_a, lane & ~(int)rlf) : ra_a, wstride, racc, 0u,
                                rlf, lane);
        racc[0] = T(0);
        rcur = kc;
      }
#pragma unroll
      for (int it = 0; it < VPT; ++it) racc[0] += sum[it][0];
    } else if (ra >= 0) {
#pragma unroll
      for (int it = 0; it < VPT; ++it) {
        const uint32_t kc = (uint32_t)sld_s32(ki32 + 4u * (uint32_t)(ra * kMaxIter + mi[it]));
        if (kc != rcur) {
          const uint32_t ra_a = win32 + (rkt + rcur) * (uint32_t)sizeof(T);
          CaseScatter<T, CB>::run(rlf != 0u ? __shfl_sync(kFull, ra_a, lane & ~(int)rlf) : ra_a, wstride, racc, 0u,
                                  rlf, lane);
#pragma unroll
          for (int cl = 0; cl < CB; ++cl) racc[cl] = T(0);
          rcur = kc;
        }
#pragma unroll
        for (int cl = 0; cl < CB; ++cl) racc[cl] += sum[it][cl];
      }
    }
    if (VPT > 1 && ja >= 0 && !jiter) {
      // a key that ignores the iteration: one accumulator for all vectors
#pragma unroll
      for (int it = 0; it < VPT; ++it)
#pragma unroll
        for (int j = 0; j < VEC; ++j) jacc[0][j] += f[it][0][j];
    } else if (ja >= 0) {
#pragma unroll
      for (int it = 0; it < VPT; ++it)
#pragma unroll
        for (int j = 0; j < VEC; ++j) jacc[it][j] += f[it][0][j];
    }
    // output scatters, reduced over the lanes that share the key
    for (int i = n_in; i < n_live; ++i) {
      if (i == ra || i == ja) continue;
      const int32_t md = sld_s32(lp32 + (uint32_t)i * (uint32_t)sizeof(LivePort));
      const uint32_t kti = (uint32_t)ktld(i);
      const uint32_t lf = (uint32_t)(md >> 3) & 31u;
      if (VPT > 1 && CB == 1 && !(md & (kModeInChunk | kModeStore))) {
        // the thread's vectors of this chunk share the key: add them first,
        // then one reduction over the lanes
        uint32_t k = kti;
        if (md & kModeIter) k += (uint32_t)sld_s32(ki32 + 4u * (uint32_t)(i * kMaxIter + mi[0]));
        const uint32_t k0 = win32 + k * (uint32_t)sizeof(T);
        if ((md & 3) == 0) {
          T v = T(0);
#pragma unroll
          for (int it = 0; it < VPT; ++it) v += sum[it][0];
          v = lane_reduce(v, lf);
          if (act[0] && (lane & lf) == 0u && v != T(0)) sred_add(k0, v);
        } else if (bfv[0] != T(0)) {
          const int4 dv = sld_v4s32(lp32 + (uint32_t)i * (uint32_t)sizeof(LivePort) + 16u);
          T fs[VEC];
#pragma unroll
          for (int j = 0; j < VEC; ++j) {
            fs[j] = f[0][0][j];
#pragma unroll
            for (int it = 1; it < VPT; ++it) fs[j] += f[it][0][j];
          }
          const uint32_t kg = lf != 0u ? __shfl_sync(kFull, k0, lane & ~(int)lf) : k0;
          scatter_vec(kg, fs, lf, lane, act[0], dv);
        }
        continue;
      }
      uint32_t ka[VPT];
#pragma unroll
      for (int it = 0; it < VPT; ++it) {
        uint32_t k = kti;
        if (md & kModeIter) k += (uint32_t)sld_s32(ki32 + 4u * (uint32_t)(i * kMaxIter + mi[it]));
        ka[it] = win32 + k * (uint32_t)sizeof(T);
      }
      if ((md & 3) == 0) {
        if (CB == 1) {
          T v[VPT];
#pragma unroll
          for (int it = 0; it < VPT; ++it) v[it] = sum[it][0];
          lane_reduce_n<T, VPT>(v, lf);
#pragma unroll
          for (int it = 0; it < VPT; ++it)
            if (act[it] && (lane & lf) == 0u && v[it] != T(0)) sred_add(ka[it], v[it]);
        } else {
#pragma unroll
          for (int it = 0; it < VPT; ++it) {
            const uint32_t kg = lf != 0u ? __shfl_sync(kFull, ka[it], lane & ~(int)lf) : ka[it];
            CaseScatter<T, CB>::run(kg, wstride, sum[it], 0u, lf, lane);
          }
        }
      } else if (md & kModeStore) {
        // every entry of the block has a key of its own: store, no
        // reduction, zeros included (the window is not zeroed beforehand)
#pragma unroll
        for (int it = 0; it < VPT; ++it)
#pragma unroll
          for (int cl = 0; cl < CB; ++cl)
            if (act[it]) sst_vec(ka[it] + (uint32_t)cl * wstride, f[it][cl]);
      } else {
        const int4 dv = sld_v4s32(lp32 + (uint32_t)i * (uint32_t)sizeof(LivePort) + 16u);
#pragma unroll
        for (int it = 0; it < VPT; ++it) {
          const uint32_t kg = lf != 0u ? __shfl_sync(kFull, ka[it], lane & ~(int)lf) : ka[it];
#pragma unroll
          for (int cl = 0; cl < CB; ++cl)
            if (bfv[cl] != T(0)) scatter_vec(kg + (uint32_t)cl * wstride, f[it][cl], lf, lane, act[it], dv);
        }
      }
    }
    if (a.calib != nullptr) {
#pragma unroll
      for (int it = 0; it < VPT; ++it)
        if (act[it]) {
#pragma unroll
          for (int cl = 0; cl < CB; ++cl)
            if (cl < ncb) VecT<T>::stg(a.calib + (int64_t)(cb0 + cl) * a.calib_stride + w.off + o0[it], f[it][cl]);
        }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(s.empty + st);
  }
  // average over the consumer warps of the time spent waiting for chunks
  if (a.trace != nullptr && lane == 0)
    atomicAdd(reinterpret_cast<unsigned long long*>(a.trace + (int64_t)s.misc[2] * kTraceSlots + 6),
              (unsigned long long)(waited / (NT / 32)));
  if (!__all_sync(kFull, ok)) return false;
  // flush the register accumulators (inactive lanes hold zeros)
  if (ra >= 0) {
    const uint32_t ra_a = win32 + (rkt + rcur) * (uint32_t)sizeof(T);
    CaseScatter<T, CB>::run(rlf != 0u ? __shfl_sync(kFull, ra_a, lane & ~(int)rlf) : ra_a, wstride, racc, 0u, rlf,
                            lane);
  }
  if (ja >= 0) {
    const uint32_t kt = (uint32_t)ktld(ja);
    const uint32_t lf = (uint32_t)(lp[ja].mode >> 3) & 31u;
    const int4 dv = make_int4(lp[ja].dvec[0], lp[ja].dvec[1], lp[ja].dvec[2], lp[ja].dvec[3]);
    const int dva[4] = {dv.x, dv.y, dv.z, dv.w};
    const bool lead = (lane & lf) == 0u;
    const int nit = jiter ? VPT : 1;  // (one accumulator when the key ignores the iteration)
#pragma unroll
    for (int it = 0; it < VPT; ++it) {
      if (it >= nit || it >= (w.n + NT * VEC - 1) / (NT * VEC)) break;  // iteration never reached
      const uint32_t k = kt + (uint32_t)sld_s32(ki32 + 4u * (uint32_t)(ja * kMaxIter + it));
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        const T v = lane_reduce(jacc[it][j], lf);
        if (lead && v != T(0)) sred_add(win32 + (k + (uint32_t)dva[j]) * (uint32_t)sizeof(T), v);
      }
    }
  }
  return ok;
}

// Stream the chunks of one item entry by entry (any cardinalities; the block
// may start inside a vector).
template <typename T, int CB>
__device__ __forceinline__ bool stream_generic(const PropArgs<T>& a, const Smem& s, const DevStage& S,
                                               const DevItem& w, int ncb, int cb0, const T (&bfv)[CB],
                                               T (&tot)[CB], RingPos& rp) {
  constexpr int NT = consumers_for(CB);
  constexpr int VEC = VecT<T>::N;
  constexpr int VPT = chunk_bytes_for(CB) / (16 * NT);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t RS = (uint32_t)a.ring, CH = (uint32_t)a.chunk;
  const uint32_t ring32 = smem_u32(s.ring), win32 = smem_u32(s.win);
  const int64_t a0 = w.off / VEC * VEC, a1 = (w.off + w.n + VEC - 1) / VEC * VEC;
  const int nchunks = (int)((a1 - a0 + CH - 1) / CH);
  const int np = S.np, nin = S.nin;
  bool ok = true;
  for (int ci = 0; ci < nchunks; ++ci, rp.advance(RS)) {
    const uint32_t st = rp.st;
    // the warp leaves together (its lanes reduce with shuffles below)
    if (!__all_sync(kFull, mbar_wait(s.full + st, rp.ph, a.err, s.misc, a.wait_ns))) {
      ok = false;
      break;
    }
    {
      const uint32_t sb = ring32 + st * CH * (uint32_t)sizeof(T);
      const int64_t cstart = a0 + (int64_t)ci * CH;
      const int nvec = (int)(min((int64_t)CH, a1 - cstart) / VEC);
#pragma unroll
      for (int it = 0; it < VPT; ++it) {
        if (it * NT + warp * 32 >= nvec) break;  // warp-uniform
        const int vi = it * NT + tid;
        const bool act = vi < nvec;
        T x[VEC];
        if (act) {
          sld_vec(sb + (uint32_t)vi * (VEC * (uint32_t)sizeof(T)), x);
        } else {
#pragma unroll
          for (int j = 0; j < VEC; ++j) x[j] = T(0);
        }
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
          const int64_t e = cstart + (int64_t)vi * VEC + j;
          const bool valid = act && e >= w.off && e < w.off + w.n;
          const uint32_t o = valid ? (uint32_t)(e - w.off) : 0u;
#pragma unroll
          for (int cl = 0; cl < CB; ++cl) {
            if (cl >= ncb) break;
            if (bfv[cl] == T(0)) continue;
            T f = valid ? x[j] * bfv[cl] : T(0);
            const int no = s.nobs[cl];
            for (int ei = 0; ei < no; ++ei) {
              const int4 ob = s.obs[cl * a.max_k + ei];
              if (digit_of(o, s.pos[ob.x]) != (uint32_t)ob.z) f = T(0);
            }
            const uint32_t W = win32 + (uint32_t)(cl * a.win_max) * (uint32_t)sizeof(T);
            for (int pi = 0; pi < nin; ++pi) {
              const DevPort& P = s.port[pi];
              if (P.K <= 1) continue;
              f *= sld<T>(W + (uint32_t)(P.win + key_of<false>(o, s.fld + P.f0, P.nf)) * (uint32_t)sizeof(T));
            }
            tot[cl] += f;
            for (int pi = nin; pi < np; ++pi) {
              const DevPort& P = s.port[pi];
              if (P.K <= 1) continue;
              add_combined<T>(W + (uint32_t)P.win * (uint32_t)sizeof(T), key_of<false>(o, s.fld + P.f0, P.nf), f, lane);
            }
            if (a.calib != nullptr && valid) a.calib[(int64_t)(cb0 + cl) * a.calib_stride + e] = f;
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(s.empty + st);
  }
  return ok;
}

// One work item (its buffer prepared by the control warp).  Every consumer
// thread runs every barrier; the result is uniform over the consumers.
template <typename T, int CB>
__device__ __forceinline__ bool process_item(const PropArgs<T>& a, const Smem& s, const DevItem& w, uint32_t b,
                                             RingPos& rp, uint32_t& sigk) {
  constexpr int NT = consumers_for(CB);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const DevStage S = *s.stage;
  const int cb0 = a.case0 + w.cbk * CB;
  const int ncb = min(CB, a.case0 + a.n_cases - cb0);
  const uint32_t eb = (uint32_t)w.block * (uint32_t)S.B;  // block start inside the clique
  const bool fast = S.bits >= 0;
  const int idx_item = s.misc[2];
  uint64_t* tr = a.trace != nullptr ? a.trace + (int64_t)idx_item * kTraceSlots : nullptr;

  // fast path: the ports with windows (inputs first) and their key tables:
  // precomputed in the stage's blob for one case; computed here for a case
  // block (iteration m covers block offsets [m, m + 1) * consumers * VEC)
  if constexpr (CB > 1) {
    constexpr int VEC = VecT<T>::N;
    if (fast) {
      LivePort* lp = reinterpret_cast<LivePort*>(s.live);
      const int mi = (w.n + NT * VEC - 1) / (NT * VEC);
      int li = 0;
      for (int pi = 0; pi < S.np; ++pi) {
        const DevPort& P = s.port[pi];
        if (P.K <= 1) continue;
        if (tid == li) {
          LivePort L;
          L.mode = (P.vmode & 3) | ((P.iter_dep & 1) ? kModeIter : 0) | ((P.iter_dep & 2) ? kModeChunk : 0) |
                   ((P.iter_dep & 4) ? kModeInChunk : 0) | ((P.vmode & kVmodeStore) ? kModeStore : 0) |
                   (int32_t)((P.lane_free & 31u) << 3);
          L.port = pi;
          L.win = P.win;
          L.pad = 0;
          for (int j = 0; j < 4; ++j) L.dvec[j] = P.dvec[j];
          lp[li] = L;
        }
        s.kt[li * NT + tid] = (int)(key_of<true>((uint32_t)tid * VEC, s.fld + P.f0, P.nf) + (uint32_t)P.win);
        for (int m = tid; m < mi; m += NT)
          s.kiter[li * kMaxIter + m] = (int)key_of<true>((uint32_t)m * NT * VEC, s.fld + P.f0, P.nf);
        ++li;
      }
    }
    consumer_sync<NT>();
  }
  // stream the block
  if (tr != nullptr && tid == 0) tr[3] = global_ns();
  T bfv[CB], tot[CB];
  bool any_obs = false;
#pragma unroll
  for (int cl = 0; cl < CB; ++cl) {
    bfv[cl] = cl < ncb ? (T)s.bf[cl] : T(0);
    tot[cl] = T(0);
    if (cl < ncb && s.nobs[cl] > 0) any_obs = true;
  }
  const bool sok = fast ? stream_fast<T, CB>(a, s, w, ncb, cb0, S.n_in_live, S.n_live, S.live_off, kiter_off(S),
                                              kt_off(S), any_obs, bfv, tot, rp)
                        : stream_generic<T, CB>(a, s, S, w, ncb, cb0, bfv, tot, rp);
  if (!consumer_all<NT>(sok)) {
    if (tid == 0) {
      atomicExch(a.err, 1);
      s.misc[0] = 1;
    }
    return false;
  }
  if (tr != nullptr && tid == 0) tr[4] = global_ns();

  // block totals (stage total, block-constant outputs); windows that are not
  // bulk-reduced by the signalling lane
  // (lanes reduce in the element type -- FP64 issue is scarce on this part;
  // the warps' partials are added in double)
#pragma unroll
  for (int cl = 0; cl < CB; ++cl) {
    const T v = warp_sum(tot[cl]);
    if (lane == 0) s.red[cl * (NT / 32) + warp] = (double)v;
  }
  consumer_sync<NT>();
  // One case: the block total goes to the signalling lane through the
  // buffer's block-factor slot (read by nothing else once the block has
  // streamed), which adds it to the stage total and the block-constant
  // outputs: the consumers then need no global fence.  A case block adds
  // its totals here.
  bool wrote_global = false;
  if (tid < ncb) {
    // four independent chains (FP64 latency is long on this part)
    static_assert((NT / 32) % 4 == 0, "consumer warps in fours");
    double t4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < NT / 32; i += 4)
#pragma unroll
      for (int q = 0; q < 4; ++q) t4[q] += s.red[tid * (NT / 32) + i + q];
    const double t = (t4[0] + t4[1]) + (t4[2] + t4[3]);
    if constexpr (CB == 1) {
      s.bf[tid] = t;
    } else {
      const int cs = cb0 + tid;
      T* row = a.msg + (int64_t)cs * a.msg_stride;
      if (t != 0.0) {
        wrote_global = true;
        for (int pi = S.nin; pi < S.np; ++pi) {
          const DevPort& P = s.port[pi];
          if (P.K > 1) continue;
          const uint32_t key = fast ? key_of<true>(eb, s.fld + P.f0, P.nf) : key_of<false>(eb, s.fld + P.f0, P.nf);
          atomicAdd(row + P.tab + key, (T)t);
        }
        atomicAdd(a.sums + (int64_t)cs * 2 * a.n_cliques + S.sum_slot, t);
      }
    }
  }
  for (int pi = S.nin; pi < S.np; ++pi) {
    const DevPort& P = s.port[pi];
    if (P.K <= 1 || bulk_window<T>(S, P)) continue;
    const uint32_t kb = fast ? key_of<true>(eb, s.fld + P.f0, P.nf) : key_of<false>(eb, s.fld + P.f0, P.nf);
    const uint32_t win32 = smem_u32(s.win);
    for (int cl = 0; cl < ncb; ++cl) {
      T* dst = a.msg + (int64_t)(cb0 + cl) * a.msg_stride + P.tab + kb;
      const uint32_t src = win32 + (uint32_t)(cl * a.win_max + P.win) * (uint32_t)sizeof(T);
      for (int i = tid; i < P.K; i += NT) {
        const T v = sld<T>(src + (uint32_t)i * (uint32_t)sizeof(T));
        if (v != T(0)) {
          atomicAdd(dst + i, v);
          wrote_global = true;
        }
      }
    }
  }
  // Every thread's global additions above (case-block totals, windows the
  // bulk unit cannot reduce) are made visible GPU-wide by the thread itself
  // before the hand-over: the signalling lane's fence orders only what it
  // wrote, and the item counts as done once it publishes.  Likewise every
  // thread's shared-memory writes to the output windows are ordered before
  // the bulk unit (the async proxy) reads them.
  if (wrote_global) __threadfence();
  fence_proxy_async();
  consumer_sync<NT>();
  if (tid == 0) {
    if (tr != nullptr) tr[5] = global_ns();
    if (!hand_over(s, sigk, make_int4(w.stage, w.cbk, (int)b, idx_item), a.err)) {
      atomicExch(a.err, 1);
      s.misc[0] = 1;
    }
  }
  return true;
}

template <typename T, int CB>
__device__ __forceinline__ void consumer(const PropArgs<T>& a, const Smem& s0) {
  constexpr int NT = consumers_for(CB);
  RingPos rp;         // ring position of the next chunk (the producer's order)
  uint32_t sigk = 0;  // items handed to the signalling lane (thread 0)
  for (uint32_t slot = 0;; ++slot) {
    const uint32_t b = slot & 1u;
    const bool ok = consumer_all<NT>(mbar_wait(s0.pfull + b, (slot >> 1) & 1u, a.err, s0.misc, a.wait_ns));
    if (!ok) {
      if (threadIdx.x == 0) {
        atomicExch(a.err, 1);
        s0.misc[0] = 1;
      }
      break;
    }
    const ItemInfo& inf = s0.info[b];
    const DevItem w = inf.w;
    if (w.stage < 0) {
      if (threadIdx.x == 0) hand_over(s0, sigk, make_int4(-1, 0, 0, -1), a.err);
      break;
    }
    if (!inf.ok) {
      if (threadIdx.x == 0) {
        atomicExch(a.err, 1);
        s0.misc[0] = 1;
      }
      break;
    }
    if (threadIdx.x == 0) {
      s0.misc[2] = inf.idx;
      if (a.trace != nullptr) {
        uint32_t smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        a.trace[(int64_t)inf.idx * kTraceSlots] = smid;
        a.trace[(int64_t)inf.idx * kTraceSlots + 1] = global_ns();
      }
    }
    consumer_sync<NT>();
    if (!process_item<T, CB>(a, with_buffer(s0, b), w, b, rp, sigk)) break;
  }
}

template <typename T, int CB>
__global__ void __launch_bounds__(consumers_for(CB) + kControlThreads, ctas_per_sm_for(CB)) k_propagate(const PropArgs<T> a) {
  constexpr int NT = consumers_for(CB);
  extern __shared__ __align__(128) unsigned char smem[];
  const SmemLayout L(CB, a.ring, a.chunk, a.max_k, a.max_ports, a.blob_max, a.win_max, (int)sizeof(T));
  const Smem s = carve(smem, L, a.ring, CB, a.max_k, a.max_ports, a.win_max, (int)sizeof(T));
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.ring; ++i) {
      mbar_init(s.full + i, 1);
      mbar_init(s.empty + i, NT / 32);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(s.ifull + i, 1);
      mbar_init(s.bfull + i, 1);
      mbar_init(s.pfull + i, 1);
      mbar_init(s.wfree + i, 1);
    }
    for (int i = 0; i < kSig; ++i) {
      mbar_init(s.sfull + i, 1);
      mbar_init(s.sempty + i, 1);
    }
    s.misc[0] = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (a.span != nullptr && threadIdx.x == 0) atomicMin(a.span, (unsigned long long)global_ns());
  if (threadIdx.x >= NT) {
    // control warps: each role has a warp of its own, so no role's waits
    // (a blocking bulk-group wait, a sleeping poll) hold up another
    const int cw = (threadIdx.x - NT) >> 5, l = threadIdx.x & 31;
    if (cw == 0) {
      if (l == 0) producer<T>(a, s);
    } else if (cw == 1) {
      if (l == 0) signaller<T, CB>(a, s);
    } else {
      prep_lanes<T, CB>(a, s);
    }
    __syncwarp();
  } else {
    consumer<T, CB>(a, s);
  }
  __syncthreads();
  if (a.span != nullptr && threadIdx.x == 0) atomicMax(a.span + 1, (unsigned long long)global_ns());
}

// Normalised marginals (a warp per variable, binned from its source table)
// and log Z(e) (the last CTA along x), per case (y).
// Warp-wide product of (pn, pd) mantissa pairs (each in [0.5, 1)) with
// their binary exponents: every lane ends with the warp's result, the
// numerator's exponent summed into en and the denominator's into ed.
__device__ __forceinline__ void mul_reduce(double& pn, double& pd, long long& en, long long& ed) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double qn = __shfl_xor_sync(kFull, pn, o), qd = __shfl_xor_sync(kFull, pd, o);
    const long long qen = __shfl_xor_sync(kFull, en, o), qed = __shfl_xor_sync(kFull, ed, o);
    en += qen;
    ed += qed;
    pn = split_exp(pn * qn, en);
    pd = split_exp(pd * qd, ed);
  }
}

constexpr int kFinStates = 8;   // variables of at most this many states: one pass over the table
constexpr int kFinUnroll = 8;   // table loads per lane in flight

template <typename T>
__global__ void __launch_bounds__(256) k_finalize(const FinalArgs<T> a) {
  const int cs = a.case0 + (int)blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* row = a.msg + (int64_t)cs * a.msg_stride;
  const double* sums = a.sums + (int64_t)cs * 2 * a.n_cliques;
  if (blockIdx.x == gridDim.x - 1) {
    // log Z = sum_c (log sigma_c - log |S_c|) + log Delta_root, as the log of
    // a product: mantissas multiplied, binary exponents summed (both read
    // off the bits), over the CTA's threads, then two logarithms in all
    // (FP64 throughput per SM is small on this part: one log per clique
    // costs more than the rest of the finalisation)
    __shared__ double pn_s[8], pd_s[8];
    __shared__ long long en_s[8], ed_s[8];
    __shared__ int zero_s[8];
    double pn = 1.0, pd = 1.0;
    long long en = 0, ed = 0;
    bool zero = false;
    int terms = 0;
    for (int c = 1 + tid; c < a.n_cliques; c += 256) {
      const double sg = sums[c];
      if (!(sg > 0.0)) {
        zero = true;
        continue;
      }
      pn *= split_exp(sg, en);
      pd *= split_exp((double)a.sep_size[c], ed);
      if (++terms == 256) {   // (a product of 256 mantissas stays above 2^-256)
        pn = split_exp(pn, en);
        pd = split_exp(pd, ed);
        terms = 0;
      }
    }
    pn = split_exp(pn, en);
    pd = split_exp(pd, ed);
    mul_reduce(pn, pd, en, ed);
    zero = __any_sync(kFull, zero);
    if (lane == 0) {
      pn_s[warp] = pn;
      pd_s[warp] = pd;
      en_s[warp] = en;
      ed_s[warp] = ed;
      zero_s[warp] = zero;
    }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < 8; ++w) {
        en += en_s[w];
        ed += ed_s[w];
        pn = split_exp(pn * pn_s[w], en);
        pd = split_exp(pd * pd_s[w], ed);
        zero = zero || zero_s[w];
      }
      const double R = sums[a.n_cliques];  // the root's distribute total
      if (zero || !(R > 0.0)) {
        atomicOr(&a.status[cs], kStatusZero);
        a.logz_out[cs] = -INFINITY;
      } else {
        a.logz_out[cs] = log(pn) - log(pd) + (double)(en - ed) * 0.69314718055994530942 + log(R);
      }
    }
    return;
  }
  const int v = (int)blockIdx.x * 8 + warp;
  if (v >= a.n_vars) return;
  const VarSrc src = a.vs[v];
  double* out = a.marg_out + (int64_t)cs * a.marg_total + src.moff;
  const T* tab = row + src.off;
  if (src.card <= kFinStates && src.size <= 2 * 32 * kFinUnroll) {
    // small tables, one pass: every state's partial sum at once (the loads
    // of all states in flight together), then one reduction each.  (Per
    // element it adds into every state's sum under a predicate: FP64 work
    // that only small tables can afford on this part.)
    double b[kFinStates];
#pragma unroll
    for (int x = 0; x < kFinStates; ++x) b[x] = 0.0;
    // (eight loads per lane in flight: the tables come from L2)
    for (int j0 = lane; j0 < src.size; j0 += 32 * kFinUnroll) {
      T val[kFinUnroll];
#pragma unroll
      for (int u = 0; u < kFinUnroll; ++u) {
        const int j = j0 + 32 * u;
        val[u] = j < src.size ? tab[j] : T(0);
      }
#pragma unroll
      for (int u = 0; u < kFinUnroll; ++u) {
        const int x = ((j0 + 32 * u) / src.st) % src.card;
#pragma unroll
        for (int y = 0; y < kFinStates; ++y)
          if (y == x) b[y] += (double)val[u];
      }
    }
    double z = 0.0;
#pragma unroll
    for (int x = 0; x < kFinStates; ++x) {
      if (x < src.card) b[x] = warp_sum(b[x]);
      z += b[x];
    }
    if (lane < src.card_out) {
      double bx = b[0];
#pragma unroll
      for (int y = 1; y < kFinStates; ++y)
        if (y == lane) bx = b[y];
      out[lane] = z > 0.0 ? bx / z : NAN;
    }
    return;
  }
  // larger tables: a pass per state (one FP64 addition per entry), eight
  // loads per lane in flight; z is the sum of the states' sums, and lane x
  // keeps the sum of state x until z is known
  const int per = src.size / src.card;  // entries holding one state
  double z = 0.0, mine = 0.0;
  for (int x = 0; x < src.card; ++x) {
    double b = 0.0;
    for (int q0 = lane; q0 < per; q0 += 32 * kFinUnroll) {
      T val[kFinUnroll];
#pragma unroll
      for (int u = 0; u < kFinUnroll; ++u) {
        const int qq = q0 + 32 * u;
        const int hi = qq / src.st, lo = qq - hi * src.st;
        val[u] = qq < per ? tab[(int64_t)(hi * src.card + x) * src.st + lo] : T(0);
      }
#pragma unroll
      for (int u = 0; u < kFinUnroll; ++u) b += (double)val[u];
    }
    b = warp_sum(b);
    z += b;
    if (x == lane) mine = b;
  }
  if (src.card <= 32) {
    if (lane < src.card_out) out[lane] = z > 0.0 ? mine / z : NAN;
    return;
  }
  // more than 32 states: each state's sum again, now that z is known
  for (int x = 0; x < src.card_out; ++x) {
    double b = 0.0;
    for (int q0 = lane; q0 < per; q0 += 32 * kFinUnroll) {
      T val[kFinUnroll];
#pragma unroll
      for (int u = 0; u < kFinUnroll; ++u) {
        const int qq = q0 + 32 * u;
        const int hi = qq / src.st, lo = qq - hi * src.st;
        val[u] = qq < per ? tab[(int64_t)(hi * src.card + x) * src.st + lo] : T(0);
      }
#pragma unroll
      for (int u = 0; u < kFinUnroll; ++u) b += (double)val[u];
    }
    b = warp_sum(b);
    if (lane == 0) out[x] = z > 0.0 ? b / z : NAN;
  }
}

// ---- calibrated-clique read-out ---------------------------------------------
// Both read-outs normalise with partial sums (one per CTA of a first pass)
// that every CTA of the gather adds up.  Scratch of the allocation-free
// read-out: the partials in a file-scope array.  Every call shares it
// (calls that overlap on the GPU race); it lives as long as the library is
// loaded on a device.
__device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks];

// Pass 1: CTA b sums entries [b * E, (b + 1) * E) of the table into partials[b]
// (every slot in use is overwritten, so nothing needs clearing).
template <typename T>
__global__ void __launch_bounds__(256) k_clique_partials(const T* p, int64_t n, double* partials) {
  __shared__ double red[8];
  const int64_t e0 = (int64_t)blockIdx.x * kNoAllocPerBlock;
  const int64_t e1 = min(n, e0 + kNoAllocPerBlock);
  double s = 0.0;
  for (int64_t i = e0 + threadIdx.x; i < e1; i += 256) s += (double)p[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    partials[blockIdx.x] = t;
  }
}

// Pass 2: every CTA adds the partials (at most kNoAllocMaxBlocks), then
// writes its share of the normalised table in the caller's listed order.
template <typename T>
__global__ void __launch_bounds__(256) k_clique_gather_partials(const T* p, CliqueOut co, const double* partials,
                                                                int nb, double* out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) s += partials[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double z = 0.0;
  for (int i = 0; i < 8; ++i) z += red[i];
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < co.n; u += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = u, src = 0;
    for (int i = co.k - 1; i >= 0; --i) {
      const int64_t d = rem % co.lcard[i];
      rem /= co.lcard[i];
      src += d * co.pst[i];
    }
    out[u] = z > 0.0 ? (double)p[src] / z : NAN;
  }
}

// The dynamic shared-memory opt-in of a propagation kernel instance, once per
// device (a process may load trees on several devices).
std::mutex g_attr_mu;

template <typename T, int CB>
cudaError_t set_attrs_once() {
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (!done[dev]) {
    e = cudaFuncSetAttribute(k_propagate<T, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_budget(dev, 1));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_propagate<T, CB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    done[dev] = true;
  }
  return cudaSuccess;
}

}  // namespace

int32_t smem_budget(int device, int ctas_per_sm) {
  int blk = 0, sm = 0, rsv = 0;
  if (cudaDeviceGetAttribute(&blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return 48 * 1024;
  if (ctas_per_sm <= 1) return blk;
  if (cudaDeviceGetAttribute(&sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess) return 48 * 1024;
  cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, device);
  return std::min(blk, sm / ctas_per_sm - rsv);
}

template <typename T>
cudaError_t launch_propagate(const PropArgs<T>& a, int cb, int grid, int smem, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (cb <= 1) {
    if ((e = set_attrs_once<T, 1>()) != cudaSuccess) return e;
    k_propagate<T, 1><<<grid, consumers_for(1) + kControlThreads, smem, s>>>(a);
  } else if (cb <= 4) {
    if ((e = set_attrs_once<T, 4>()) != cudaSuccess) return e;
    k_propagate<T, 4><<<grid, consumers_for(4) + kControlThreads, smem, s>>>(a);
  } else {
    if ((e = set_attrs_once<T, 8>()) != cudaSuccess) return e;
    k_propagate<T, 8><<<grid, consumers_for(8) + kControlThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_finalize(const FinalArgs<T>& a, cudaStream_t s) {
  if (a.n_cases <= 0) return cudaSuccess;
  dim3 grid((a.n_vars + 7) / 8 + 1, a.n_cases);
  k_finalize<T><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_get_clique(const T* calib_clique, const CliqueOut& co, double* out_dev, double* sum_dev,
                              cudaStream_t s) {
  // the normalising sum as partial sums of kNoAllocPerBlock entries each
  // (sum_dev holds one per block), which every gather block adds up
  const int nb = (int)((co.n + kNoAllocPerBlock - 1) / kNoAllocPerBlock);
  if (nb == 0) return cudaSuccess;
  k_clique_partials<T><<<nb, 256, 0, s>>>(calib_clique, (int64_t)co.n, sum_dev);
  const int blocks = (int)std::min<int64_t>(1024, (co.n + 255) / 256);
  k_clique_gather_partials<T><<<blocks, 256, 0, s>>>(calib_clique, co, sum_dev, nb, out_dev);
  return cudaGetLastError();
}

// Device address of the read-out scratch on the current device, looked up
// once per device (with that device current) and cached.
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[kNoAllocMaxDevices] = {};

cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_get_clique_noalloc(const T* calib_clique, const CliqueOut& co, double* out_dev, cudaStream_t s) {
  double* partials = nullptr;
  cudaError_t e = noalloc_scratch(&partials);
  if (e != cudaSuccess) return e;
  const int nb = (int)((co.n + kNoAllocPerBlock - 1) / kNoAllocPerBlock);
  k_clique_partials<T><<<nb, 256, 0, s>>>(calib_clique, (int64_t)co.n, partials);
  const int blocks = (int)std::min<int64_t>(1024, (co.n + 255) / 256);
  k_clique_gather_partials<T><<<blocks, 256, 0, s>>>(calib_clique, co, partials, nb, out_dev);
  return cudaGetLastError();
}

template cudaError_t launch_get_clique_noalloc<float>(const float*, const CliqueOut&, double*, cudaStream_t);
template cudaError_t launch_get_clique_noalloc<double>(const double*, const CliqueOut&, double*, cudaStream_t);
template cudaError_t launch_propagate<float>(const PropArgs<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_propagate<double>(const PropArgs<double>&, int, int, int, cudaStream_t);
template cudaError_t launch_finalize<float>(const FinalArgs<float>&, cudaStream_t);
template cudaError_t launch_finalize<double>(const FinalArgs<double>&, cudaStream_t);
template cudaError_t launch_get_clique<float>(const float*, const CliqueOut&, double*, double*, cudaStream_t);
template cudaError_t launch_get_clique<double>(const double*, const CliqueOut&, double*, double*, cudaStream_t);

}  // namespace jt

// Case-lane propagation kernel (FP32, power-of-two cliques).
//
// The same persistent schedule as k_propagate (Algorithm 4: collect,
// Algorithm 2, then distribute, Algorithm 3, over work items that are blocks
// of clique tables), with the evidence cases of an item laid across the lanes
// of a warp: lane l of every consumer warp computes case l of the item's
// block of kCaseLanes cases.  Per entry x of the streamed block and case l,
//
//   collect, clique c (Eq. 2):
//       f_l(x) = phi_c(x) E_l(x) prod_g mu_g,l[key_g(x)]
//       u_c,l[key_p(x)] += f_l(x)
//   distribute, clique c (Eq. 3, then Eq. 2 towards every child):
//       f_l(x) = phi_c(x) E_l(x) prod_g mu_g,l[key_g(x)] rho_c,l[key_p(x)]
//       delta_g,l[key_g(x)] += f_l(x),   joint_c,l[key_priv(x)] += f_l(x)
//
// Every lane of a warp handles the same x at the same time, so the table
// value phi_c(x) is one broadcast shared-memory load for the 32 cases, the
// keys are common to them, and each lane gathers from and reduces into its
// own column of case-minor windows (row = key, 32 cases of 4 bytes): loads
// and reductions of a warp touch 32 consecutive words, conflict-free, and no
// value crosses lanes.  Messages live in global memory in the same case-minor
// order (a slab of 32 cases: [entry][case]), so a window moves with a single
// bulk copy or bulk reduction.
//
// Per-case factors that are constant over a block (the child messages'
// normalisation |S_g|/sigma_g, block-constant inputs, evidence on digits above
// the block) are applied once per item to the reduced windows instead of per
// entry.  Evidence E_l on a digit inside the block needs no per-entry work when
// the digit's variable belongs to an input port of the stage: the message on
// that port was computed under the same evidence and is already zero where
// the state differs (a child's collect message, or the ratio of the own
// separator, whose old table is then zero, with 0/0 := 0).  The remaining
// in-block observed digits (private variables, and in the collect pass the
// parent-separator variables no child shares) are masked per lane.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "jt_device.cuh"

namespace jt {
namespace {

constexpr int NT = 512;        // consumer threads
constexpr int NW = NT / 32;    // consumer warps
static_assert(NW * kClSlice == 2048, "a chunk of 2048 entries is the consumers' slices");
static_assert(NW * kClTiles <= 64, "slot table");

__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 dup(float x) { return make_float2(x, x); }

// Shared-memory load / reduction at a register address plus a compile-time
// offset (one instruction, no address arithmetic).
template <int OFF>
__device__ __forceinline__ float sld_at(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF));
  return v;
}
template <int OFF>
__device__ __forceinline__ void sred_at(uint32_t a, float v) {
  asm volatile("red.shared.add.f32 [%0+%1], %2;" ::"r"(a), "n"(OFF), "f"(v) : "memory");
}
// The 32 entries of a tile at consecutive window rows (keys key + e).
template <int E>
struct IdentRows {
  __device__ __forceinline__ static void gather_mul(uint32_t at, float2 (&f)[16]) {
    IdentRows<E - 2>::gather_mul(at, f);
    f[(E - 2) / 2] = mul2(f[(E - 2) / 2], make_float2(sld_at<(E - 2) * kClRow>(at), sld_at<(E - 1) * kClRow>(at)));
  }
  __device__ __forceinline__ static void reduce(uint32_t at, const float2 (&f)[16]) {
    IdentRows<E - 2>::reduce(at, f);
    sred_at<(E - 2) * kClRow>(at, f[(E - 2) / 2].x);
    sred_at<(E - 1) * kClRow>(at, f[(E - 2) / 2].y);
  }
};
template <>
struct IdentRows<0> {
  __device__ __forceinline__ static void gather_mul(uint32_t, float2 (&)[16]) {}
  __device__ __forceinline__ static void reduce(uint32_t, const float2 (&)[16]) {}
};

// Output reductions that first add up the values of a tile whose keys
// coincide: VF holds the vector bits (tile-offset bits 2, 3, 4 as bits 0, 1,
// 2) the port's key ignores, so vector v | u adds into vector v's rows for
// every u inside VF, and only vectors outside VF reduce into the window --
// 8 >> popcount(VF) of them instead of 8.  VF = 0 (no combining) is correct
// for every port, so only the common patterns get their own instance: joint
// ports over a variable on the lowest digit (VF = 7), and keys over a digit
// on tile-offset bits 2-3 (VF = 4) or bit 4 (VF = 3).
template <int VF>
__device__ __forceinline__ void red_vectors(uint32_t at, uint32_t kv, const float (&vs)[8]) {
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    if (v & VF) continue;
    float a = vs[v];
#pragma unroll
    for (int u = 1; u < 8; ++u)
      if ((u & ~VF) == 0) a += vs[v | u];
    sred_add(at + (uint32_t)sld_s32(kv + 4u * v), a);
  }
}
template <int VF>
__device__ __forceinline__ void red_entries(uint32_t at, uint32_t kv, const int4 dv, const float2 (&f)[16]) {
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    if (v & VF) continue;
    float2 a = f[2 * v], b = f[2 * v + 1];
#pragma unroll
    for (int u = 1; u < 8; ++u)
      if ((u & ~VF) == 0) {
        a = add2(a, f[2 * (v | u)]);
        b = add2(b, f[2 * (v | u) + 1]);
      }
    const uint32_t av = at + (uint32_t)sld_s32(kv + 4u * v);
    sred_add(av + (uint32_t)dv.x, a.x);
    sred_add(av + (uint32_t)dv.y, a.y);
    sred_add(av + (uint32_t)dv.z, b.x);
    sred_add(av + (uint32_t)dv.w, b.y);
  }
}

// The four distinct sums of a tile for an output whose key depends only on
// entry bits 0-1 (a joint over the lowest digit; the slot is encoded in the
// class): each entry position summed over the tile's eight vectors.
__device__ __forceinline__ void tile_sums(const float2 (&f)[16], float (&o)[4]) {
  float2 a = f[0], b = f[1];
#pragma unroll
  for (int v = 1; v < 8; ++v) {
    a = add2(a, f[2 * v]);
    b = add2(b, f[2 * v + 1]);
  }
  o[0] = a.x;
  o[1] = a.y;
  o[2] = b.x;
  o[3] = b.y;
}
__device__ __forceinline__ void acc4(float (&r)[4], const float (&o)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) r[i] += o[i];
}

// Shared-memory carve-up of a case-lane CTA.  The common fields serve the
// producer; per buffer: `obs` holds (V, M) per case, `bf` the block factor per
// case (then the block totals), `win` the case-minor windows.
__device__ __forceinline__ Smem carve_cl(unsigned char* smem, const SmemLayoutCL& L, int ring_n, int win_max) {
  Smem s{};
  s.full = reinterpret_cast<uint64_t*>(smem + L.bar);
  s.empty = s.full + ring_n;
  s.ifull = s.empty + ring_n;
  s.bfull = s.ifull + 2;
  s.pfull = s.bfull + 2;
  s.wfree = s.pfull + 2;
  s.sfull = s.wfree + 2;
  s.sempty = s.sfull + kSig;
  s.info = reinterpret_cast<ItemInfo*>(smem + L.info);
  s.sig = reinterpret_cast<int4*>(smem + L.sig);
  s.blob0 = smem + L.blob;
  s.blob_stride = (uint32_t)L.blob_bytes;
  s.obs = reinterpret_cast<int4*>(smem + L.ev);
  s.nobs = nullptr;
  s.bf = reinterpret_cast<double*>(smem + L.bf);
  s.pval = nullptr;
  s.win = smem + L.win;
  s.red = reinterpret_cast<double*>(smem + L.red);
  s.misc = reinterpret_cast<int*>(smem + L.misc);
  s.kiter = nullptr;
  s.live = nullptr;
  s.kt = nullptr;
  s.ring = smem + L.ring;
  s.obs_b = (uint32_t)(kCaseLanes * 16);
  s.nobs_b = 0;
  s.bf_b = (uint32_t)(kCaseLanes * 8);
  s.pval_b = 0;
  s.win_b = (uint32_t)(win_max * kClRow);
  return s;
}

// ---- control warp 2: preparation of the next item (lane = case) ------------
// Evidence (digits above the block into the case's block factor, uncovered
// digits inside it into the case's mask), the output windows zeroed, the
// dependency wait, the child-message windows by bulk copy (one per port: the
// slab rows are already case-minor), the per-case factors, and the ratio
// windows of the own separator, rho = delta (sigma_c / Delta_parent) / u with
// 0/0 := 0 (Eq. 3 and its zero rule).
__device__ __forceinline__ void prep_cl(const PropArgs<float>& a, const Smem& s0) {
  constexpr int U = 16;  // ratio rows per lane per round (their loads in flight together)
  const int l = (int)(threadIdx.x & 31);
  for (uint32_t slot = 0;; ++slot) {
    const uint32_t b = slot & 1u, par = (slot >> 1) & 1u;
    if (!__all_sync(kFull, mbar_wait(s0.ifull + b, par, a.err, s0.misc, a.wait_ns))) break;
    ItemInfo& inf = s0.info[b];
    const DevItem w = inf.w;
    if (w.stage < 0) {
      __syncwarp();
      if (l == 0) mbar_arrive(s0.pfull + b);
      break;
    }
    if (!__all_sync(kFull, mbar_wait(s0.bfull + b, par, a.err, s0.misc, a.wait_ns))) break;
    const Smem s = with_buffer(s0, b);
    const DevStage S = *s.stage;
    const int cb0 = a.case0 + w.cbk * kCaseLanes;
    const int ncb = min(kCaseLanes, a.case0 + a.n_cases - cb0);
    const bool valid = l < ncb;
    const int cs = cb0 + l;
    const uint32_t eb = (uint32_t)w.block * (uint32_t)S.B;
    float* slab = a.msg + (int64_t)cb0 * a.msg_stride;
    uint64_t* tr = a.trace != nullptr ? a.trace + (int64_t)inf.idx * kTraceSlots : nullptr;
    if (tr != nullptr && l == 0) tr[11] = global_ns();
    // evidence of this lane's case
    double bf = valid ? 1.0 : 0.0;
    uint32_t V = 0, M = 0;
    if (valid) {
      const int16_t* evr = a.ev + (int64_t)cs * a.n_vars;
      // the case's states of kEB positions are loaded before any is used
      // (independent loads in flight together)
      constexpr int kEB = 8;
      for (int i0 = 0; i0 < S.k; i0 += kEB) {
        int sts[kEB];
#pragma unroll
        for (int j = 0; j < kEB; ++j) sts[j] = i0 + j < S.k ? (int)evr[s.pos[i0 + j].var] : -1;
#pragma unroll
        for (int j = 0; j < kEB; ++j) {
          const int i = i0 + j;
          const int st = sts[j];
          if (i >= S.k || st < 0) continue;
          const DevPos& P = s.pos[i];
          if (st >= P.card_ev) {
            atomicOr(&a.status[cs], kStatusBadState);
            continue;
          }
          const int inside = max(0, min(P.cb, S.bits - P.sh));
          const uint32_t lo_m = (1u << inside) - 1u;
          const uint32_t hi_d = (eb >> P.sh) & ((1u << P.cb) - 1u);
          if (hi_d != ((uint32_t)st & ~lo_m)) {
            bf = 0.0;
          } else if (lo_m != 0u && !((S.covered >> i) & 1u)) {
            M |= lo_m << P.sh;
            V |= ((uint32_t)st & lo_m) << P.sh;
          }
        }
      }
    }
    s.obs[l] = make_int4((int)V, (int)M, 0, 0);
    // output windows start at zero (32 lanes x 16 bytes = four rows a store)
    const uint32_t win32 = smem_u32(s.win);
    {
      const float z[4] = {0.f, 0.f, 0.f, 0.f};
      for (int pi = S.nin; pi < S.np; ++pi) {
        const DevPort& P = s.port[pi];
        if (P.K <= 1) continue;
        const uint32_t base = win32 + (uint32_t)P.win * kClRow, bytes = (uint32_t)P.K * kClRow;
        for (uint32_t o = (uint32_t)l * 16u; o < bytes; o += 512u) sst_vec(base + o, z);
      }
    }
    bool dok = true;
    if (S.ndep > 0) dok = await_deps(a.deps + S.dep0, S.ndep, a.done, a.n_cb, w.cbk, a.err, s.misc, l, 32, kFull, a.wait_ns);
    if (tr != nullptr && l == 0) tr[10] = global_ns();
    if (dok) {
      uint32_t bulk = 0;
      for (int pi = 0; pi < S.nin; ++pi) {
        const DevPort& P = s.port[pi];
        if (P.K > 1 && P.kind == kPortMu) bulk += (uint32_t)P.K * kClRow;
      }
      if (l == 0) mbar_expect_tx_only(s.pfull + b, bulk);
      __syncwarp();
      if (bulk > 0) {
        fence_proxy_async_all();  // the messages were written by other CTAs (bulk reductions)
        // lane l copies the l-th such window: the lanes find theirs first,
        // then compute the window keys and issue the copies together (a
        // case-lane stage has at most as many ports as a warp has lanes)
        int mine = -1, n = 0;
        for (int pi = 0; pi < S.nin; ++pi) {
          const DevPort& P = s.port[pi];
          if (P.K <= 1 || P.kind != kPortMu) continue;
          if (n++ == l) mine = pi;
        }
        if (mine >= 0) {
          const DevPort& P = s.port[mine];
          const uint32_t kb = key_of<true>(eb, s.fld + P.f0, P.nf);
          bulk_g2s(s.win + (size_t)P.win * kClRow, slab + (int64_t)(P.tab + kb) * kCaseLanes,
                   (uint32_t)P.K * kClRow, s.pfull + b);
        }
      }
      // per-case factor: the child messages' scales and block-constant inputs.
      // The loads of kPB ports are issued together (one round trip to L2 per
      // group instead of one per port; nothing uses a loaded value before
      // the group's last load is issued), and the factors are formed in
      // FP32: the consumers apply the block factor in FP32, and FP64
      // divisions are slow on this part.
      if (valid) {
        constexpr int kPB = 8;
        const double* sums = a.sums + (int64_t)cs * 2 * a.n_cliques;
        float bff = 1.f;
        for (int p0 = 0; p0 < S.nin; p0 += kPB) {
          double t0[kPB], t1[kPB];  // stage totals
          float e0[kPB], e1[kPB];   // slab entries
#pragma unroll
          for (int j = 0; j < kPB; ++j) {
            t0[j] = t1[j] = 0.0;
            e0[j] = e1[j] = 0.f;
            const int pi = p0 + j;
            if (pi >= S.nin) continue;
            const DevPort& P = s.port[pi];
            if (P.kind == kPortMu) {
              t0[j] = __ldcg(sums + P.other);
              if (P.K <= 1) {
                const uint32_t key = key_of<true>(eb, s.fld + P.f0, P.nf);
                e0[j] = __ldcg(slab + (int64_t)(P.tab + key) * kCaseLanes + l);
              }
            } else if (P.K <= 1) {
              const uint32_t key = key_of<true>(eb, s.fld + P.f0, P.nf);
              t0[j] = __ldcg(sums + P.other);
              t1[j] = __ldcg(sums + a.n_cliques + P.other2);
              e0[j] = __ldcg(slab + (int64_t)(P.tab + key) * kCaseLanes + l);
              e1[j] = __ldcg(slab + (int64_t)(a.delta_off + P.tab + key) * kCaseLanes + l);
            }
          }
#pragma unroll
          for (int j = 0; j < kPB; ++j) {
            const int pi = p0 + j;
            if (pi >= S.nin) continue;
            const DevPort& P = s.port[pi];
            const float s0 = (float)t0[j], s1 = (float)t1[j];
            float v = 1.f;
            if (P.kind == kPortMu) {
              v = s0 > 0.f ? (float)P.size / s0 : 0.f;
              if (P.K <= 1) v *= e0[j];
            } else if (P.K <= 1) {
              v = (s1 > 0.f && e0[j] > 0.f) ? e1[j] * (s0 / s1) / e0[j] : 0.f;
            }
            bff *= v;
          }
        }
        bf *= (double)bff;
      }
      // ratio windows of the own separator, row by row (lane = case)
      for (int pi = 0; pi < S.nin; ++pi) {
        const DevPort& P = s.port[pi];
        if (P.K <= 1 || P.kind != kPortRho) continue;
        const uint32_t kb = key_of<true>(eb, s.fld + P.f0, P.nf);
        float sc = 0.f;
        if (valid) {
          const double* sums = a.sums + (int64_t)cs * 2 * a.n_cliques;
          const float sgc = (float)__ldcg(sums + P.other), dp = (float)__ldcg(sums + a.n_cliques + P.other2);
          sc = dp > 0.f ? sgc / dp : 0.f;
        }
        const float* ur = slab + (int64_t)(P.tab + kb) * kCaseLanes + l;
        const float* dr = slab + (int64_t)(a.delta_off + P.tab + kb) * kCaseLanes + l;
        const uint32_t dst = win32 + (uint32_t)P.win * kClRow + 4u * (uint32_t)l;
        for (int i0 = 0; i0 < P.K; i0 += U) {
          float u[U], d[U];
#pragma unroll
          for (int r = 0; r < U; ++r) {
            const int ii = min(i0 + r, P.K - 1);
            u[r] = __ldcg(ur + (int64_t)ii * kCaseLanes);
            d[r] = __ldcg(dr + (int64_t)ii * kCaseLanes);
          }
#pragma unroll
          for (int r = 0; r < U; ++r)
            if (i0 + r < P.K) sst<float>(dst + (uint32_t)(i0 + r) * kClRow, u[r] > 0.f ? d[r] * sc / u[r] : 0.f);
        }
      }
    }
    s.bf[l] = bf;
    if (l == 0) inf.ok = dok ? 1 : 0;
    __syncwarp();
    if (tr != nullptr && l == 0) tr[2] = global_ns();
    if (l == 0) {
      if (!dok) mbar_expect_tx_only(s.pfull + b, 0u);
      mbar_arrive(s.pfull + b);  // completes once the bulk window bytes have landed
    }
    if (!dok) break;  // the consumers see ok = 0 and stop
  }
}

// ---- control warp 1: the signalling warp (lane = case) ---------------------
// For each finished item: add each case's block total (left in the buffer's
// block-factor slot) to its stage total and to the block-constant outputs
// (lane l for case l), add the output windows into the slab rows with one
// bulk reduction per port (lane 0), wait until they completed, make every
// lane's writes visible GPU-wide, count the block as done, and free the
// item's buffer.
__device__ __forceinline__ void signaller_cl(const PropArgs<float>& a, const Smem& s0) {
  const int l = (int)(threadIdx.x & 31);
  for (uint32_t k = 0;; ++k) {
    const uint32_t sl = k % kSig;
    if (!__all_sync(kFull, mbar_wait(s0.sfull + sl, (k / kSig) & 1u, a.err, s0.misc, a.wait_ns))) break;
    const int4 g = s0.sig[sl];   // stage, case block, buffer, item index
    __syncwarp();
    if (l == 0) mbar_arrive(s0.sempty + sl);
    if (g.x < 0) break;
    const uint32_t b = (uint32_t)g.z;
    const Smem s = with_buffer(s0, b);
    const DevStage& S = *s.stage;
    const DevItem& w = s0.info[b].w;
    const uint32_t eb = (uint32_t)w.block * (uint32_t)S.B;
    const int cb0 = a.case0 + g.y * kCaseLanes;
    const int ncb = min(kCaseLanes, a.case0 + a.n_cases - cb0);
    float* slab = a.msg + (int64_t)cb0 * a.msg_stride;
    if (l < ncb) {
      const double t = s.bf[l];
      if (t != 0.0) {
        for (int pi = S.nin; pi < S.np; ++pi) {
          const DevPort& P = s.port[pi];
          if (P.K > 1) continue;
          const uint32_t key = key_of<true>(eb, s.fld + P.f0, P.nf);
          atomicAdd(slab + (int64_t)(P.tab + key) * kCaseLanes + l, (float)t);
        }
        atomicAdd(a.sums + (int64_t)(cb0 + l) * 2 * a.n_cliques + S.sum_slot, t);
      }
    }
    if (l == 0) {
      // the consumers' window writes (generic proxy) before the bulk reads
      fence_proxy_async();
      bool any = false;
      for (int pi = S.nin; pi < S.np; ++pi) {
        const DevPort& P = s.port[pi];
        if (P.K <= 1) continue;
        const uint32_t kb = key_of<true>(eb, s.fld + P.f0, P.nf);
        bulk_reduce_add(slab + (int64_t)(P.tab + kb) * kCaseLanes, s.win + (size_t)P.win * kClRow,
                        (uint32_t)P.K * kClRow);
        any = true;
      }
      if (any) {
        bulk_commit();
        bulk_wait_all();
        fence_proxy_async_all();
      }
    }
    // every lane's additions visible GPU-wide before the block counts as done
    __threadfence();
    __syncwarp();
    if (l == 0) {
      atomicAdd(a.done + (int64_t)g.x * a.n_cb + g.y, 1);
      if (a.trace != nullptr && g.w >= 0) a.trace[(int64_t)g.w * kTraceSlots + 9] = global_ns();
      mbar_arrive(s0.wfree + b);
    }
  }
}

// ---- consumers -------------------------------------------------------------

// A digit of a padded plan at one of its added states (packed as in
// DevStage::holes): every table entry with it is zero.
__device__ __forceinline__ bool added_state(uint32_t x, uint32_t h) {
  return h != 0u && ((x >> (h & 31u)) & ((1u << ((h >> 5) & 31u)) - 1u)) >= (h >> 10);
}

// Stream one item: every warp takes its slice of each chunk in tiles of 32
// entries; per tile a lane holds the 32 products of its case in registers
// (as 16 pairs, multiplied and added two at a time).  A tile of a padded
// plan whose digits above the tile include an added state holds only zero
// entries and is skipped: it would add nothing.
template <bool HOLES>
__device__ __forceinline__ bool stream_cl(const PropArgs<float>& a, const Smem& s, const DevItem& w, int ncb,
                                          int cb0, int n_in, int n_live, float bfl, float& tot, RingPos& rp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t RS = (uint32_t)a.ring;
  const int CH = a.chunk;
  const uint32_t ring32 = smem_u32(s.ring);
  const uint32_t cp32 = smem_u32(s.stage) + (uint32_t)s.stage->live_off;   // the stage's port tables (blob)
  const uint32_t lane4 = smem_u32(s.win) + 4u * (uint32_t)lane;           // the lane's column of the windows
  const int nchunks = (w.n + CH - 1) / CH;
  // this lane's evidence mask: tile-level bits (>= 5), per vector (2-4), per entry (0-1)
  const int4 evm = s.obs[lane];
  const uint32_t V = (uint32_t)evm.x, M = (uint32_t)evm.y;
  const uint32_t VT = V & ~31u, MT = M & ~31u;
  const bool ev_t = __any_sync(kFull, MT != 0u);
  const bool ev_v = __any_sync(kFull, (M & 28u) != 0u);
  const bool ev_e = __any_sync(kFull, (M & 3u) != 0u);
  uint32_t mvb = 0;   // bit v: the lane's case admits vector v of a tile
#pragma unroll
  for (int v = 0; v < 8; ++v) mvb |= ((((uint32_t)(4 * v)) ^ V) & M & 28u) == 0u ? 1u << v : 0u;
  const float2 mA01 = make_float2(((0u ^ V) & M & 3u) == 0u ? 1.f : 0.f, ((1u ^ V) & M & 3u) == 0u ? 1.f : 0.f);
  const float2 mA23 = make_float2(((2u ^ V) & M & 3u) == 0u ? 1.f : 0.f, ((3u ^ V) & M & 3u) == 0u ? 1.f : 0.f);
  float* calib = (a.calib != nullptr && lane < ncb) ? a.calib + (int64_t)(cb0 + lane) * a.calib_stride + w.off : nullptr;
  const uint32_t h0 = s.stage->holes[0], h1 = s.stage->holes[1], h2 = s.stage->holes[2];
  const uint32_t xb = (uint32_t)(w.off - s.stage->base_off);   // the block's first entry in its clique
  // register-accumulated outputs (tile-only keys), reduced after the block
  float racc[kClRegSlots][4];
#pragma unroll
  for (int r = 0; r < kClRegSlots; ++r)
#pragma unroll
    for (int i = 0; i < 4; ++i) racc[r][i] = 0.f;
  bool ok = true;
  for (int ci = 0; ci < nchunks; ++ci, rp.advance(RS)) {
    const uint32_t st = rp.st;
    if (!__all_sync(kFull, mbar_wait(s.full + st, rp.ph, a.err, s.misc, a.wait_ns))) {
      ok = false;
      break;
    }
    const int nch = min(CH, w.n - ci * CH);
    const uint32_t sb = ring32 + st * (uint32_t)CH * 4u;
#pragma unroll 1
    for (int t = 0; t < kClTiles; ++t) {
      // tile positions interleave over the warps: a short block still keeps
      // every warp busy
      const int slot = warp + NW * t;
      const int ot = 32 * slot;                 // tile offset in the chunk
      if (ot >= nch) break;                     // warp-uniform
      if (HOLES && h0 != 0u) {
        const uint32_t x = xb + (uint32_t)(ci * CH + ot);
        if (added_state(x, h0) || added_state(x, h1) || added_state(x, h2)) continue;
      }
      float2 f[16];
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        float x[4];
        sld_vec(sb + (uint32_t)(ot + 4 * v) * 4u, x);
        f[2 * v] = make_float2(x[0], x[1]);
        f[2 * v + 1] = make_float2(x[2], x[3]);
      }
      // the lane's evidence mask and block factor (every product carries the
      // case's per-block factor, so the reduced windows need no rescaling)
      {
        const uint32_t oa = (uint32_t)(ci * CH + ot);
        const float sc = (!ev_t || ((oa ^ VT) & MT) == 0u) ? bfl : 0.f;
        if (ev_e) {
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            const float2 m = dup((mvb >> v) & 1u ? sc : 0.f);
            f[2 * v] = mul2(f[2 * v], mul2(mA01, m));
            f[2 * v + 1] = mul2(f[2 * v + 1], mul2(mA23, m));
          }
        } else if (ev_v) {
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            const float2 m = dup((mvb >> v) & 1u ? sc : 0.f);
            f[2 * v] = mul2(f[2 * v], m);
            f[2 * v + 1] = mul2(f[2 * v + 1], m);
          }
        } else {
          const float2 m = dup(sc);
#pragma unroll
          for (int i = 0; i < 16; ++i) f[i] = mul2(f[i], m);
        }
      }
      // inputs: gather the lane's own case column and multiply
#pragma unroll 1
      for (int li = 0; li < n_in; ++li) {
        const uint32_t pb = cp32 + (uint32_t)li * (uint32_t)sizeof(CLPort);
        const int cls = sld_s32(pb + offsetof(CLPort, cls));
        const uint32_t at = (uint32_t)sld_s32(pb + offsetof(CLPort, kchunk) + 4u * (uint32_t)ci) +
                            (uint32_t)sld_s32(pb + offsetof(CLPort, kslot) + 4u * (uint32_t)slot) + lane4;
        if (cls & kClIdent) {
          IdentRows<32>::gather_mul(at, f);
        } else if (cls & kClEntry) {
          const int4 kv0 = sld_v4s32(pb + offsetof(CLPort, kvec));
          const int4 kv1 = sld_v4s32(pb + offsetof(CLPort, kvec) + 16u);
          const int4 dv = sld_v4s32(pb + offsetof(CLPort, dvec));
          const int kv[8] = {kv0.x, kv0.y, kv0.z, kv0.w, kv1.x, kv1.y, kv1.z, kv1.w};
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            const uint32_t av = at + (uint32_t)kv[v];
            const float2 g01 = make_float2(sld<float>(av + (uint32_t)dv.x), sld<float>(av + (uint32_t)dv.y));
            const float2 g23 = make_float2(sld<float>(av + (uint32_t)dv.z), sld<float>(av + (uint32_t)dv.w));
            f[2 * v] = mul2(f[2 * v], g01);
            f[2 * v + 1] = mul2(f[2 * v + 1], g23);
          }
        } else if (cls & kClVector) {
          const int4 kv0 = sld_v4s32(pb + offsetof(CLPort, kvec));
          const int4 kv1 = sld_v4s32(pb + offsetof(CLPort, kvec) + 16u);
          const int kv[8] = {kv0.x, kv0.y, kv0.z, kv0.w, kv1.x, kv1.y, kv1.z, kv1.w};
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            const float2 g = dup(sld<float>(at + (uint32_t)kv[v]));
            f[2 * v] = mul2(f[2 * v], g);
            f[2 * v + 1] = mul2(f[2 * v + 1], g);
          }
        } else {
          const float2 g = dup(sld<float>(at));
#pragma unroll
          for (int i = 0; i < 16; ++i) f[i] = mul2(f[i], g);
        }
      }
      // per-vector and tile sums (the stage total and the coarser outputs)
      float vs[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const float2 p = add2(f[2 * v], f[2 * v + 1]);
        vs[v] = p.x + p.y;
      }
      const float ts = ((vs[0] + vs[1]) + (vs[2] + vs[3])) + ((vs[4] + vs[5]) + (vs[6] + vs[7]));
      tot += ts;
      // outputs: reduce into the lane's own case column
#pragma unroll 1
      for (int li = n_in; li < n_live; ++li) {
        const uint32_t pb = cp32 + (uint32_t)li * (uint32_t)sizeof(CLPort);
        const int cls = sld_s32(pb + offsetof(CLPort, cls));
        // (the variant that skips tiles has no registers to spare: there a
        // marked output reduces per tile like the others)
        if (const int rs = HOLES ? 0 : (cls >> kClRegShift) & 3) {
          float o[4];
          tile_sums(f, o);
          acc4(racc[0], o);
          continue;
        }
        const uint32_t at = (uint32_t)sld_s32(pb + offsetof(CLPort, kchunk) + 4u * (uint32_t)ci) +
                            (uint32_t)sld_s32(pb + offsetof(CLPort, kslot) + 4u * (uint32_t)slot) + lane4;
        if (cls & kClIdent) {
          IdentRows<32>::reduce(at, f);
        } else if (cls & (kClEntry | kClVector)) {
          const uint32_t kv = pb + offsetof(CLPort, kvec);
          const int vf = (~sld_s32(pb + offsetof(CLPort, dep)) >> 2) & 7;
          if (cls & kClEntry) {
            const int4 dv = sld_v4s32(pb + offsetof(CLPort, dvec));
            if (vf == 7) red_entries<7>(at, kv, dv, f);
            else if (vf == 4) red_entries<4>(at, kv, dv, f);
            else red_entries<0>(at, kv, dv, f);
          } else {
            if (vf == 3) red_vectors<3>(at, kv, vs);
            else if (vf == 4) red_vectors<4>(at, kv, vs);
            else if (vf == 7) red_vectors<7>(at, kv, vs);
            else red_vectors<0>(at, kv, vs);
          }
        } else {
          sred_add(at, ts);
        }
      }
      // calibrated table (JT_MATERIALIZE_CLIQUES), in the permuted layout
      // of the base table
      if (calib != nullptr) {
        float* dst = calib + ci * CH + ot;
#pragma unroll
        for (int v = 0; v < 8; ++v)
          __stcs(reinterpret_cast<float4*>(dst + 4 * v),
                 make_float4(f[2 * v].x, f[2 * v].y, f[2 * v + 1].x, f[2 * v + 1].y));
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(s.empty + st);
  }
  // the register-accumulated outputs, once per item (their rows are the same
  // for every tile: chunk 0, slot 0)
  if (!HOLES && ok) {
#pragma unroll 1
    for (int li = n_in; li < n_live; ++li) {
      const uint32_t pb = cp32 + (uint32_t)li * (uint32_t)sizeof(CLPort);
      const int cls = sld_s32(pb + offsetof(CLPort, cls));
      const int rs = (cls >> kClRegShift) & 3;
      if (rs == 0) continue;
      float o[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) o[i] = racc[0][i];
      const uint32_t at = (uint32_t)sld_s32(pb + offsetof(CLPort, kchunk)) +
                          (uint32_t)sld_s32(pb + offsetof(CLPort, kslot)) + lane4;
      const uint32_t kv = pb + offsetof(CLPort, kvec);
      const int4 dv = sld_v4s32(pb + offsetof(CLPort, dvec));
      const uint32_t av = at + (uint32_t)sld_s32(kv);
      sred_add(av + (uint32_t)dv.x, o[0]);
      sred_add(av + (uint32_t)dv.y, o[1]);
      sred_add(av + (uint32_t)dv.z, o[2]);
      sred_add(av + (uint32_t)dv.w, o[3]);
    }
  }
  return __all_sync(kFull, ok);
}

// One work item (its buffer prepared by the control warp).  Every consumer
// thread runs every barrier; the result is uniform over the consumers.
template <bool HOLES>
__device__ __forceinline__ bool process_item_cl(const PropArgs<float>& a, const Smem& s, const DevItem& w, uint32_t b,
                                                RingPos& rp, uint32_t& sigk) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const DevStage& S = *s.stage;
  const int cb0 = a.case0 + w.cbk * kCaseLanes;
  const int ncb = min(kCaseLanes, a.case0 + a.n_cases - cb0);
  const int idx_item = s.misc[2];
  uint64_t* tr = a.trace != nullptr ? a.trace + (int64_t)idx_item * kTraceSlots : nullptr;
  if (tr != nullptr && tid == 0) tr[3] = global_ns();
  const float bfl = (float)s.bf[lane];
  float tot = 0.f;
  const bool sok = stream_cl<HOLES>(a, s, w, ncb, cb0, S.n_in_live, S.n_live, bfl, tot, rp);
  if (!consumer_all<NT>(sok)) {
    if (tid == 0) {
      atomicExch(a.err, 1);
      s.misc[0] = 1;
    }
    return false;
  }
  if (tr != nullptr && tid == 0) tr[4] = global_ns();
  s.red[lane * NW + warp] = (double)tot;
  consumer_sync<NT>();
  // the block total of each case goes to the signalling lane through the
  // buffer's block-factor slot (read by nothing else once the block has
  // streamed); the lane adds it to the stage total and the block-constant
  // outputs, so no consumer writes global memory here.  The window writes are
  // ordered before the bulk unit reads them.
  if (tid < kCaseLanes) {
    double t = 0.0;
    for (int i = 0; i < NW; ++i) t += s.red[tid * NW + i];
    s.bf[tid] = tid < ncb ? t : 0.0;
  }
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

template <bool HOLES>
__device__ __forceinline__ void consumer_cl(const PropArgs<float>& a, const Smem& s0) {
  RingPos rp;
  uint32_t sigk = 0;
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
    if (!process_item_cl<HOLES>(a, with_buffer(s0, b), w, b, rp, sigk)) break;
  }
}

// HOLES: the schedule is a padded plan's, whose all-zero tiles are skipped.
template <bool HOLES>
__global__ void __launch_bounds__(NT + kControlThreads, 1) k_propagate_cl(const PropArgs<float> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SmemLayoutCL L(a.ring, a.chunk, a.blob_max, a.win_max);
  const Smem s = carve_cl(smem, L, a.ring, a.win_max);
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.ring; ++i) {
      mbar_init(s.full + i, 1);
      mbar_init(s.empty + i, NW);
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
    const int cw = (threadIdx.x - NT) >> 5, l = threadIdx.x & 31;
    if (cw == 0) {
      if (l == 0) producer<float>(a, s);
    } else if (cw == 1) {
      signaller_cl(a, s);
    } else {
      prep_cl(a, s);
    }
    __syncwarp();
  } else {
    consumer_cl<HOLES>(a, s);
  }
  __syncthreads();
  if (a.span != nullptr && threadIdx.x == 0) atomicMax(a.span + 1, (unsigned long long)global_ns());
}

// Normalised marginals and log Z(e) of the cases of a slab (blockIdx.y),
// lane = case (coalesced reads of the case-minor rows).  A CTA per variable
// (blockIdx.x; the last one computes log Z): for each state x its eight
// warps sum the source-table entries holding x (strided over the warps), the
// partial sums meet in shared memory, and warp 0 writes the bin; the bins are
// then normalised by their total.  Entries of a power-of-two table are split
// into (hi, lo) around the variable's digit by shifts.
__global__ void __launch_bounds__(256) k_finalize_cl(const FinalArgs<float> a) {
  __shared__ double red[8][32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cb0 = a.case0 + (int)blockIdx.y * kCaseLanes;
  const int ncb = min(kCaseLanes, a.case0 + a.n_cases - cb0);
  const int cs = cb0 + lane;
  const bool valid = lane < ncb;
  const float* slab = a.msg + (int64_t)cb0 * a.msg_stride;
  // blocks: groups of 8 small-source variables (a warp each), then one block
  // per other variable, then log Z
  const int g_small = (a.n_small + 7) / 8;
  const int bx = (int)blockIdx.x;
  if (bx < g_small) {
    const int i = bx * 8 + warp;
    if (i >= a.n_small || !valid) return;
    const VarSrc src = a.vs[a.var_order[i]];
    const float* tab = slab + (int64_t)src.off * kCaseLanes + lane;
    const int per = src.size / src.card;
    const bool p2 = (src.st & (src.st - 1)) == 0;
    const int sh = __ffs(src.st) - 1;
    double* out = a.marg_out + (int64_t)cs * a.marg_total + src.moff;
    // lane = case: each state's entries summed by the lane itself (rows of 32
    // cases, so a warp's loads are 128 consecutive bytes), no barrier
    double z = 0.0;
    for (int x = 0; x < src.card; ++x) {
      double b = 0.0;
#pragma unroll 8
      for (int q = 0; q < per; ++q) {
        const int h = p2 ? q >> sh : q / src.st;
        b += (double)__ldcg(tab + ((int64_t)(h * src.card + x) * src.st + (q - h * src.st)) * kCaseLanes);
      }
      z += b;
      if (x < src.card_out) out[x] = b;
    }
    for (int x = 0; x < src.card_out; ++x) out[x] = z > 0.0 ? out[x] / z : NAN;
    return;
  }
  const int v = bx - g_small < a.n_vars - a.n_small ? a.var_order[a.n_small + (bx - g_small)] : a.n_vars;
  if (v == a.n_vars) {
    if (warp != 0 || !valid) return;
    // log Z = sum_c (log sigma_c - log |S_c|) + log Delta_root, as the log of
    // a product (mantissas multiplied, binary exponents summed, both read off
    // the bits): two logarithms per case instead of two per clique
    const double* sums = a.sums + (int64_t)cs * 2 * a.n_cliques;
    double pn = 1.0, pd = 1.0;
    long long en = 0, ed = 0;
    bool zero = false;
    int terms = 0;
    for (int c = 1; c < a.n_cliques; ++c) {
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
    const double R = sums[a.n_cliques];
    if (zero || !(R > 0.0)) {
      atomicOr(&a.status[cs], kStatusZero);
      a.logz_out[cs] = -INFINITY;
    } else {
      a.logz_out[cs] = log(pn) - log(pd) + (double)(en - ed) * 0.69314718055994530942 + log(R);
    }
    return;
  }
  const VarSrc src = a.vs[v];
  const float* tab = slab + (int64_t)src.off * kCaseLanes + lane;
  const int per = src.size / src.card;
  const bool p2 = (src.st & (src.st - 1)) == 0;
  const int sh = __ffs(src.st) - 1;
  double* out = a.marg_out + (int64_t)cs * a.marg_total + src.moff;
  double z = 0.0;
  // states from card_out up are padded ones (zero in every table)
  for (int x = 0; x < src.card_out; ++x) {
    double s0 = 0.0, s1 = 0.0;
    int q = warp;
#pragma unroll 2
    for (; q + 8 < per; q += 16) {
      const int h0 = p2 ? q >> sh : q / src.st, h1 = p2 ? (q + 8) >> sh : (q + 8) / src.st;
      s0 += (double)__ldcg(tab + ((int64_t)(h0 * src.card + x) * src.st + (q - h0 * src.st)) * kCaseLanes);
      s1 += (double)__ldcg(tab + ((int64_t)(h1 * src.card + x) * src.st + (q + 8 - h1 * src.st)) * kCaseLanes);
    }
    if (q < per) {
      const int h0 = p2 ? q >> sh : q / src.st;
      s0 += (double)__ldcg(tab + ((int64_t)(h0 * src.card + x) * src.st + (q - h0 * src.st)) * kCaseLanes);
    }
    red[warp][lane] = s0 + s1;
    __syncthreads();
    if (warp == 0) {
      double b = 0.0;
      for (int w = 0; w < 8; ++w) b += red[w][lane];
      z += b;
      if (valid) out[x] = b;
    }
    __syncthreads();
  }
  if (warp == 0 && valid)
    for (int x = 0; x < src.card_out; ++x) out[x] = z > 0.0 ? out[x] / z : NAN;
}

// The dynamic shared-memory opt-in of the propagation kernel, once per device.
std::mutex g_attr_mu;
bool g_attr_done[64] = {};

cudaError_t set_attrs_cl() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (!g_attr_done[dev]) {
    for (auto k : {k_propagate_cl<false>, k_propagate_cl<true>}) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_budget(dev, 1));
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
    }
    g_attr_done[dev] = true;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_propagate_cl(const PropArgs<float>& a, int grid, int smem, bool holes, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  cudaError_t e = set_attrs_cl();
  if (e != cudaSuccess) return e;
  if (holes) k_propagate_cl<true><<<grid, NT + kControlThreads, smem, s>>>(a);
  else k_propagate_cl<false><<<grid, NT + kControlThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_finalize_cl(const FinalArgs<float>& a, cudaStream_t s) {
  if (a.n_cases <= 0) return cudaSuccess;
  dim3 grid((a.n_small + 7) / 8 + (a.n_vars - a.n_small) + 1, (a.n_cases + kCaseLanes - 1) / kCaseLanes);
  k_finalize_cl<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace jt

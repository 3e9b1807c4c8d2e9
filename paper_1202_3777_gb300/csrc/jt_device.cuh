// Device-side building blocks shared by the propagation kernels: PTX
// wrappers (shared-memory access, mbarriers, bulk copies and reductions),
// bounded waits, table keys, the shared-memory carve-up of a propagation
// CTA, and the roles every schedule shares (the producer that streams a
// block's table into the bulk-copy ring, the dependency wait, the hand-over
// of a finished item to the signalling lane).
#pragma once

#include <cstdint>

#include "jt_kernels.h"

namespace jt {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s bound on every device-side wait

template <typename T>
struct VecT;
template <>
struct VecT<float> {
  static constexpr int N = 4;
  __device__ static void lds(const float* p, float (&x)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  }
  __device__ static void stg(float* p, const float (&x)[4]) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(x[0], x[1], x[2], x[3]));
  }
};
template <>
struct VecT<double> {
  static constexpr int N = 2;
  __device__ static void lds(const double* p, double (&x)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    x[0] = v.x; x[1] = v.y;
  }
  __device__ static void stg(double* p, const double (&x)[2]) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(x[0], x[1]));
  }
};

// ---- PTX helpers ----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// Explicit shared-memory accesses by 32-bit shared address, so the hot
// loops never fall back to generic addressing.
template <typename T>
__device__ __forceinline__ T sld(uint32_t a);
template <>
__device__ __forceinline__ float sld<float>(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
template <>
__device__ __forceinline__ double sld<double>(uint32_t a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int32_t sld_s32(uint32_t a) {
  int32_t v;
  asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int4 sld_v4s32(uint32_t a) {
  int4 v;
  asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t sld_u16(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sld_vec(uint32_t a, float (&x)[4]) {
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]) : "r"(a));
}
__device__ __forceinline__ void sld_vec(uint32_t a, double (&x)[2]) {
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(x[0]), "=d"(x[1]) : "r"(a));
}
__device__ __forceinline__ void sst_vec(uint32_t a, const float (&x)[4]) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x[0]), "f"(x[1]), "f"(x[2]), "f"(x[3])
               : "memory");
}
__device__ __forceinline__ void sst_vec(uint32_t a, const double (&x)[2]) {
  asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(x[0]), "d"(x[1]) : "memory");
}
template <typename T>
__device__ __forceinline__ void sst(uint32_t a, T v);
template <>
__device__ __forceinline__ void sst<float>(uint32_t a, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v));
}
template <>
__device__ __forceinline__ void sst<double>(uint32_t a, double v) {
  asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(v));
}
__device__ __forceinline__ void sred_add(uint32_t a, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void sred_add(uint32_t a, double v) {
  asm volatile("red.shared.add.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx_only(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Bulk reduction shared -> global (add), tracked by the bulk async-group of
// the issuing thread.
__device__ __forceinline__ void bulk_reduce_add(float* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_reduce_add(double* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_all() { asm volatile("fence.proxy.async;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int32_t ld_acquire(const int32_t* p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int32_t ld_relaxed(const int32_t* p) {
  int32_t v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Named barrier of the NT consumer threads (the producer warp never joins it).
template <int NT>
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); }
// Consumer barrier that also ANDs a predicate over every consumer thread.
template <int NT>
__device__ __forceinline__ bool consumer_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(NT)
      : "memory");
  return r != 0;
}

// Wait for phase `parity` of `bar`.  False once the wait limit passed, or
// (when given) once the error word or the CTA's abort flag is set.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const int32_t* err,
                                          const volatile int* abort, uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++spins & 63u) == 0) {
      if (global_ns() - t0 > limit_ns) return false;
      if (abort != nullptr && *abort) return false;
      if (err != nullptr && ld_relaxed(err) != 0) return false;
    }
  }
  return true;
}

// n / d for n < 2^31 with m = ceil(2^32 / d): umulhi gives the quotient or
// one more; one compare corrects it.
__device__ __forceinline__ uint32_t udiv(uint32_t n, uint32_t d, uint32_t m) {
  if (d == 1u) return n;
  uint32_t q = __umulhi(n, m);
  if (q * d > n) --q;
  return q;
}

// Key of entry offset x in a small table (fields in shared memory).
template <bool POW2>
__device__ __forceinline__ uint32_t key_of(uint32_t x, const DevField* f, int nf) {
  uint32_t key = 0;
  for (int i = 0; i < nf; ++i) {
    const DevField q = f[i];
    uint32_t d;
    if (POW2) {
      d = (x >> q.sh) & ((1u << q.lb) - 1u);
    } else {
      const uint32_t t = udiv(x, (uint32_t)q.st, q.st_magic);
      d = t - udiv(t, (uint32_t)q.len, q.len_magic) * (uint32_t)q.len;
    }
    key += d * (uint32_t)q.w;
  }
  return key;
}

__device__ __forceinline__ uint32_t digit_of(uint32_t x, const DevPos& p) {
  const uint32_t t = udiv(x, (uint32_t)p.st, p.st_magic);
  return t - udiv(t, (uint32_t)p.card, p.card_magic) * (uint32_t)p.card;
}

// x = m 2^e with m in [0.5, 1), for finite x > 0, adding e to `ex`: the
// exponent field is read and replaced with integer operations (no FP64
// arithmetic); subnormal x goes through frexp.
__device__ __forceinline__ double split_exp(double x, long long& ex) {
  const long long b = __double_as_longlong(x);
  const int f = (int)((b >> 52) & 0x7FF);
  if (f == 0) {
    int k;
    const double m = frexp(x, &k);
    ex += k;
    return m;
  }
  ex += f - 1022;
  return __longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | 0x3FE0000000000000ll);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Sum over the lanes that differ from this one only in the bits of `mask`.
template <typename T>
__device__ __forceinline__ T lane_reduce(T v, uint32_t mask) {
#pragma unroll
  for (int b = 1; b < 32; b <<= 1)
    if (mask & (uint32_t)b) v += __shfl_xor_sync(kFull, v, b);
  return v;
}

// lane_reduce of N independent values at once (their shuffle chains overlap).
template <typename T, int N>
__device__ __forceinline__ void lane_reduce_n(T (&v)[N], uint32_t mask) {
#pragma unroll
  for (int b = 1; b < 32; b <<= 1)
    if (mask & (uint32_t)b) {
#pragma unroll
      for (int i = 0; i < N; ++i) v[i] += __shfl_xor_sync(kFull, v[i], b);
    }
}

// A work item as handed from the producer to the preparation lanes and the
// consumers, with its preparation status.
struct ItemInfo {
  DevItem w;
  int32_t idx;        // item index (for the optional trace)
  int32_t ok;         // preparation succeeded (dependencies met in time)
  int32_t pad[6];
};
static_assert(sizeof(ItemInfo) == 64, "item info slot");

struct Smem {
  // barriers: ring stages; per buffer b: item written (producer -> prep),
  // blob landed, item prepared (prep -> consumers, with the window copies'
  // bytes), windows flushed (signaller -> producer); signal slots
  uint64_t *full, *empty, *ifull, *bfull, *pfull, *wfree, *sfull, *sempty;
  ItemInfo* info;           // [2]
  int4* sig;                // [kSig] (stage, case block, buffer, block start)
  unsigned char* blob0;     // two descriptor blobs, blob_stride apart
  uint32_t blob_stride;
  // the current item's descriptors (inside its blob)
  const DevStage* stage;
  const DevPort* port;
  const DevField* fld;
  const DevPos* pos;
  // per-buffer state (the current item's buffer for the consumers)
  int4* obs;                // [cb][max_k] in-block observations
  int* nobs;                // [cb]
  double* bf;               // [cb] block factor
  double* pval;             // [cb][max_ports] per (case, input port) factor
  unsigned char* win;       // [cb][win_max] windows
  double* red;
  int* misc;                // [0] abort flag, [2] current item index
  // case blocks: the live ports' key tables, computed per item (one-case
  // schedules read them from the blob)
  int* kiter;               // [kMaxFastPorts][kMaxIter]
  unsigned char* live;      // [kMaxFastPorts] LivePort
  int* kt;                  // [kMaxFastPorts][consumers]
  unsigned char* ring;
  // buffer strides (bytes)
  uint32_t obs_b, nobs_b, bf_b, pval_b, win_b;
};

// Position in the bulk-copy ring: stage and the parity of its current round
// (kept incrementally: no division in the hot loop).
struct RingPos {
  uint32_t st = 0, ph = 0;
  __device__ __forceinline__ void advance(uint32_t stages) {
    if (++st == stages) {
      st = 0;
      ph ^= 1u;
    }
  }
};

__device__ __forceinline__ Smem carve(unsigned char* smem, const SmemLayout& L, int ring_n, int cb, int max_k,
                                      int max_ports, int win_max, int elem) {
  Smem s;
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
  s.stage = nullptr;
  s.port = nullptr;
  s.fld = nullptr;
  s.pos = nullptr;
  s.obs = reinterpret_cast<int4*>(smem + L.obs);
  s.nobs = reinterpret_cast<int*>(smem + L.nobs);
  s.bf = reinterpret_cast<double*>(smem + L.bf);
  s.pval = reinterpret_cast<double*>(smem + L.pval);
  s.win = smem + L.win;
  s.red = reinterpret_cast<double*>(smem + L.red);
  s.misc = reinterpret_cast<int*>(smem + L.misc);
  s.kiter = reinterpret_cast<int*>(smem + L.kiter);
  s.live = smem + L.live;
  s.kt = reinterpret_cast<int*>(smem + L.kt);
  s.ring = smem + L.ring;
  s.obs_b = (uint32_t)(cb * max_k * 16);
  s.nobs_b = (uint32_t)(cb * 4);
  s.bf_b = (uint32_t)(cb * 8);
  s.pval_b = (uint32_t)(cb * max_ports * 8);
  s.win_b = (uint32_t)(cb * win_max * elem);
  return s;
}

// The per-buffer state of buffer b, with the descriptors of the blob in it.
__device__ __forceinline__ Smem with_buffer(const Smem& s, uint32_t b) {
  Smem r = s;
  unsigned char* blob = s.blob0 + b * s.blob_stride;
  r.stage = reinterpret_cast<const DevStage*>(blob);
  r.port = reinterpret_cast<const DevPort*>(blob + sizeof(DevStage));
  r.fld = reinterpret_cast<const DevField*>(r.port + r.stage->np);
  r.pos = reinterpret_cast<const DevPos*>(r.fld + r.stage->nf);
  r.obs = reinterpret_cast<int4*>(reinterpret_cast<unsigned char*>(s.obs) + b * s.obs_b);
  r.nobs = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(s.nobs) + b * s.nobs_b);
  r.bf = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(s.bf) + b * s.bf_b);
  r.pval = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(s.pval) + b * s.pval_b);
  r.win = s.win + b * s.win_b;
  return r;
}

// ---- control warp, lane 0: the producer -----------------------------------
// Takes items from the queue into buffer slot & 1 (once the item two slots
// back has been flushed), fetches the stage's descriptor blob, and streams the
// block into the ring, running ahead of the consumers.
template <typename T>
__device__ __forceinline__ void producer(const PropArgs<T>& a, const Smem& s) {
  constexpr int VEC = VecT<T>::N;
  volatile int* abort = s.misc;
  T* ring = reinterpret_cast<T*>(s.ring);
  const uint32_t S = (uint32_t)a.ring, CH = (uint32_t)a.chunk;
  uint32_t q = 0;      // chunks issued
  uint32_t nblob = 0;  // descriptor blobs issued
  RingPos rp;
  bool ok = true;
  for (uint32_t slot = 0;; ++slot) {
    const uint32_t b = slot & 1u;
    if (slot >= 2 && !mbar_wait(s.wfree + b, ((slot >> 1) - 1) & 1u, a.err, abort, a.wait_ns)) {
      ok = false;
      break;
    }
    int it = a.n_items;
    if (!*abort && ld_relaxed(a.err) == 0) it = atomicAdd(a.queue, 1);
    ItemInfo& inf = s.info[b];
    inf.w.stage = -1;
    inf.idx = -1;
    if (it < a.n_items) {
      inf.w = a.items[it];
      inf.idx = it;
      if (a.trace != nullptr) a.trace[(int64_t)it * kTraceSlots + 7] = global_ns();
      fence_proxy_async();
      mbar_expect_tx(s.bfull + b, (uint32_t)inf.w.blob_bytes);
      bulk_g2s(s.blob0 + b * s.blob_stride, a.blobs + inf.w.blob, (uint32_t)inf.w.blob_bytes, s.bfull + b);
      ++nblob;
    }
    const DevItem w = inf.w;
    mbar_arrive(s.ifull + b);
    if (w.stage < 0) break;
    const int64_t a0 = w.off / VEC * VEC, a1 = (w.off + w.n + VEC - 1) / VEC * VEC;
    for (int64_t e = a0; e < a1; e += CH, ++q, rp.advance(S)) {
      const uint32_t st = rp.st;
      // the stage's previous round must have been released by every consumer warp
      if (q >= S && !mbar_wait(s.empty + st, rp.ph ^ 1u, a.err, abort, a.wait_ns)) {
        ok = false;
        break;
      }
      fence_proxy_async();
      const uint32_t ne = (uint32_t)min((int64_t)CH, a1 - e);
      mbar_expect_tx(s.full + st, ne * (uint32_t)sizeof(T));
      bulk_g2s(ring + (size_t)st * CH, a.base + e, ne * (uint32_t)sizeof(T), s.full + st);
    }
    if (a.trace != nullptr) a.trace[(int64_t)it * kTraceSlots + 8] = global_ns();
    if (!ok) break;
  }
  if (!ok) {
    atomicExch(a.err, 1);
    *abort = 1;
  }
  // every issued copy lands before the CTA may exit (the last chunk of each stage)
  for (uint32_t j = q > S ? q - S : 0; j < q; ++j) mbar_wait(s.full + j % S, (j / S) & 1u, nullptr, nullptr);
  for (uint32_t j = nblob > 2 ? nblob - 2 : 0; j < nblob; ++j) mbar_wait(s.bfull + (j & 1u), (j / 2) & 1u, nullptr, nullptr);
}

// Wait until every dependency of the item has all its blocks finished (one
// dependency per lane of `lanes` lanes).  False if the wait limit passed or an
// error was reported.
__device__ __forceinline__ bool await_deps(const int32_t* deps, int ndep, const int32_t* done, int n_cb, int cbk,
                                           const int32_t* err, const volatile int* abort, int lane, int lanes,
                                           unsigned mask, uint64_t limit_ns = kWaitLimitNs) {
  bool ok = true;
  for (int d = lane; d < ndep; d += lanes) {
    const int32_t stg = deps[2 * d], need = deps[2 * d + 1];
    const int32_t* ctr = done + (int64_t)stg * n_cb + cbk;
    if (ld_acquire(ctr) >= need) continue;
    const uint64_t t0 = global_ns();
    while (ld_acquire(ctr) < need) {
      if (*abort || ld_relaxed(err) != 0 || global_ns() - t0 > limit_ns) {
        ok = false;
        break;
      }
      __nanosleep(100);
    }
    if (!ok) break;
  }
  return __all_sync(mask, ok);
}

// Window copies need 16-byte aligned, 16-byte granular ranges on both sides.
template <typename T>
__device__ __forceinline__ bool bulk_window(const DevStage& S, const DevPort& P) {
  return S.bits >= 0 && ((uint32_t)P.K * (uint32_t)sizeof(T)) % 16u == 0u;
}

// Consumer thread 0: hand a finished item to the signalling lane (stage < 0
// ends it).  False if the lane did not free the slot in time.
__device__ __forceinline__ bool hand_over(const Smem& s, uint32_t& k, int4 g, const int32_t* err) {
  const uint32_t sl = k % kSig;
  if (k >= (uint32_t)kSig && !mbar_wait(s.sempty + sl, ((k / kSig) - 1) & 1u, err, s.misc)) return false;
  s.sig[sl] = g;
  mbar_arrive(s.sfull + sl);
  ++k;
  return true;
}

}  // namespace
}  // namespace jt

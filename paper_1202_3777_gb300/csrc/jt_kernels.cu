// Message kernels for Hugin propagation on sm_103a.
//
// One launch processes one tree depth ("level") of one pass for a block of
// evidence cases.  Each CTA owns a contiguous slice [t0, t1) of one clique's
// table and a block of cases, and streams the slice once with 16-byte vector
// loads.  The clique table is a matrix of rows x P columns (the columns are
// the private variables, see jt_internal.h), so per row:
//
//   collect (Algorithm 2, Eq. 2):
//       F(r)   = E_row(r) * prod_g mu_g[key_g(r)]
//       u_c[seg(r)] += F(r) * sum_col phi(r, col) * E_col(col)
//   distribute (Algorithm 3, Eq. 3):
//       G(r)   = F(r) * rho_c[seg(r)]            rho = new/old separator, 0/0 := 0
//       psi*(r, col) = G(r) * phi(r, col) * E_col(col)       (calibrated entry)
//       delta_g[key_g(r)] += sum_col psi*(r, col)             (child messages, Eq. 2)
//       joint[col] += psi*(r, col)                            (private marginals)
//
// mu_g are child collect messages normalised to mean one; E_row / E_col are
// the evidence indicators evaluated on the row / column digits.  The last CTA
// to finish a clique (ticket counter after a fence; no CTA ever waits on
// another) finalises its outgoing messages once: collect normalises u_c and
// records log(sigma); distribute turns each child message into the ratio
// rho_g and bins the separator- and joint-held marginals.
#include <cmath>
#include <cstdint>

#include "jt_kernels.h"

namespace jt {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = kLevelThreads;        // consumer threads of a level CTA
constexpr int kWarps = kThreads / 32;
constexpr int kBlock = kThreads + 32;            // + one producer warp (bulk copies)
constexpr int kVpt = 2;                          // vectors per consumer thread per chunk
constexpr int kStatusZero = 1;      // some message or the root summed to zero: P(e) = 0
constexpr int kStatusBadState = 2;  // an evidence state >= card

template <typename T>
struct VecT;
template <>
struct VecT<float> {
  static constexpr int N = 4;
  __device__ static void load(const float* p, float (&x)[4]) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  }
  __device__ static void lds(const float* p, float (&x)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  }
  __device__ static void store(float* p, const float (&x)[4]) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(x[0], x[1], x[2], x[3]));
  }
};
template <>
struct VecT<double> {
  static constexpr int N = 2;
  __device__ static void load(const double* p, double (&x)[2]) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    x[0] = v.x; x[1] = v.y;
  }
  __device__ static void lds(const double* p, double (&x)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    x[0] = v.x; x[1] = v.y;
  }
  __device__ static void store(double* p, const double (&x)[2]) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(x[0], x[1]));
  }
};

// n / d for n < 2^31 with m = ceil(2^32 / d): umulhi gives the quotient or
// one more; one compare corrects it.
__device__ __forceinline__ uint32_t udiv(uint32_t n, uint32_t d, uint32_t m) {
  if (d == 1u) return n;
  uint32_t q = __umulhi(n, m);
  if (q * d > n) --q;
  return q;
}

// digit of position p in an index x (row index for row positions, column
// index for column positions)
template <bool POW2>
__device__ __forceinline__ uint32_t digit(uint32_t x, const DevPos& p) {
  if (POW2) return (x >> p.sh) & ((1u << p.cbits) - 1u);
  const uint32_t q = udiv(x, (uint32_t)p.st, p.st_magic);
  return q - udiv(q, (uint32_t)p.card, p.card_magic) * (uint32_t)p.card;
}

template <bool POW2>
__device__ __forceinline__ uint32_t eval_key(uint32_t r, const DevField* f, int nf) {
  uint32_t key = 0;
  for (int i = 0; i < nf; ++i) {
    uint32_t x;
    if (POW2) {
      x = (r >> f[i].sh) & ((1u << f[i].lbits) - 1u);
    } else {
      const uint32_t q = udiv(r, (uint32_t)f[i].st, f[i].st_magic);
      x = q - udiv(q, (uint32_t)f[i].len, f[i].len_magic) * (uint32_t)f[i].len;
    }
    key += x * (uint32_t)f[i].w;
  }
  return key;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Add v at tab[key] for every lane of a full warp; when all lanes share the
// key the warp reduces first and issues one atomic.
template <typename T>
__device__ __forceinline__ void add_combined(T* tab, uint32_t key, T v, int lane) {
  const uint32_t k0 = __shfl_sync(kFull, key, 0);
  if (__all_sync(kFull, key == k0)) {
    v = warp_sum(v);
    if (lane == 0 && v != T(0)) atomicAdd(tab + k0, v);
  } else if (v != T(0)) {
    atomicAdd(tab + key, v);
  }
}

// Sum over a level CTA in double (all kBlock threads call; red holds >= 17 doubles).
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < kBlock / 32; ++i) t += red[i];
  return t;
}

// Shared-memory view of one CTA's tables (set up by the kernel prologue).
// ---- bulk-copy (TMA) staging: cp.async.bulk global -> shared, completed on
// an mbarrier by transaction count.  Waits are bounded by %globaltimer.
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
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
__device__ __forceinline__ void st_release(int32_t* p, int32_t v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Wait for phase `parity` of `bar`; false if it did not complete in time (or,
// with `err`, once another CTA reported an error).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const int32_t* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > kWaitLimitNs) return false;
    if (err != nullptr && ld_acquire(err) != 0) return false;
  }
  return true;
}

template <typename T>
struct CtaView {
  const DevChild* ch;
  const DevField* fld;
  const DevHome* hm;
  const DevPos* pos;
  const int2* obs;     // [cb][k] row observations
  const int2* cobs;    // [cb][k] column observations
  const int* nobs;     // [cb] row, then [cb] column counts
  const T* const* facp;
  T* const* outp;
  const T* const* rhop;
  T* const* houtp;
  T* const* jntp;
  T* win;
  T* buf;              // [stages][chunk] staging ring
  uint64_t* bar;       // [stages] "full" mbarriers (bulk-copy bytes landed)
  uint64_t* ebar;      // [stages] "empty" mbarriers (every consumer warp done)
  T* rsum;             // [cb][rowmax] row sums of the slice
  T* gsm;              // [cb][rowmax] row factors of the slice (distribute)
};

// Column evidence factor (0 or 1) of column `col` for case cl.
template <typename T, bool POW2>
__device__ __forceinline__ T colmask(const CtaView<T>& v, const SmemPlan& sp, int cl, uint32_t col) {
  const int nco = v.nobs[sp.cb + cl];
  for (int o = 0; o < nco; ++o) {
    const int2 ob = v.cobs[cl * sp.k + o];
    if (digit<POW2>(col, v.pos[ob.x]) != (uint32_t)ob.y) return T(0);
  }
  return T(1);
}

// Row factor without the parent ratio: E_row(r) prod_g mu_g[key_g(r)].
template <typename T, bool POW2, int CBMAX>
__device__ __forceinline__ void row_factor(const CtaView<T>& v, const SmemPlan& sp, int nch, int ncb, uint32_t r,
                                           T (&F)[CBMAX]) {
#pragma unroll
  for (int cl = 0; cl < CBMAX; ++cl) {
    F[cl] = T(1);
    if (cl < ncb) {
      for (int o = 0; o < v.nobs[cl]; ++o) {
        const int2 ob = v.obs[cl * sp.k + o];
        if (digit<POW2>(r, v.pos[ob.x]) != (uint32_t)ob.y) F[cl] = T(0);
      }
    }
  }
  for (int t = 0; t < nch; ++t) {
    const uint32_t key = eval_key<POW2>(r, v.fld + v.ch[t].field_rel, v.ch[t].n_field);
#pragma unroll
    for (int cl = 0; cl < CBMAX; ++cl)
      if (cl < ncb) F[cl] *= v.facp[cl * sp.n_child + t][key];
  }
}

// Geometry of one slice [t0, t1) of a clique: the table is a matrix of
// rows x P columns (jt_internal.h); the slice covers rows r_lo .. r_lo+nrow-1
// (a row cut by a slice boundary is shared through atomics).
struct SliceGeo {
  uint32_t t0, t1, P, LR, r_lo, seg_lo;
  int nrow;
};

template <bool POW2>
__device__ __forceinline__ uint32_t row_of(const DevClique& c, uint32_t e) {
  return POW2 ? (e >> c.logP) : udiv(e, (uint32_t)c.P, c.P_magic);
}
template <bool POW2>
__device__ __forceinline__ uint32_t seg_of(const DevClique& c, uint32_t r) {
  return POW2 ? (r >> c.logLR) : udiv(r, (uint32_t)c.LR, c.LR_magic);
}

template <bool POW2>
__device__ __forceinline__ SliceGeo slice_geo(const DevClique& c, uint32_t t0, uint32_t t1) {
  SliceGeo g;
  g.t0 = t0;
  g.t1 = t1;
  g.P = (uint32_t)c.P;
  g.LR = (uint32_t)c.LR;
  g.r_lo = row_of<POW2>(c, t0);
  g.nrow = (int)(row_of<POW2>(c, t1 - 1) - g.r_lo + 1);
  g.seg_lo = seg_of<POW2>(c, g.r_lo);
  return g;
}

// Rows phase before streaming (distribute): G(r) = E_row(r) prod_g mu_g[key_g(r)] rho[seg(r)].
template <typename T, bool POW2, int CBMAX>
__device__ __forceinline__ void rows_factor(const SmemPlan& sp, const DevClique& c, const CtaView<T>& v,
                                            const SliceGeo& g, int ncb, bool is_root) {
  const int tid = threadIdx.x;
  if (tid >= kThreads) return;
#pragma unroll 2
  for (int pr = tid; pr < g.nrow; pr += kThreads) {
    const uint32_t r = g.r_lo + (uint32_t)pr;
    T F[CBMAX];
    row_factor<T, POW2, CBMAX>(v, sp, c.n_child, ncb, r, F);
    const uint32_t sg = seg_of<POW2>(c, r);
#pragma unroll
    for (int cl = 0; cl < CBMAX; ++cl)
      if (cl < ncb) v.gsm[(size_t)cl * sp.rowmax + pr] = is_root ? F[cl] : F[cl] * v.rhop[cl][sg];
  }
}

// The bulk-copy ring over [t0, t1): the producer warp refills a stage once
// every consumer warp released it; consumer warps call fn(ce, cend, sb) for
// each chunk (entries [ce, cend) staged at sb) and never wait for each other.
// Chunks carry a per-CTA sequence number seq0 + ci, so stages and mbarrier
// phases continue across the CTA's items; the item prologue issued the first
// n_pre chunks.  Returns false (after letting issued copies land) if a wait
// timed out or another CTA reported an error.
template <typename T, typename Fn>
__device__ __forceinline__ bool ring_stream(const LevelArgs<T>& a, const SmemPlan& sp, const CtaView<T>& v,
                                            const T* tab, uint32_t t0, uint32_t t1, uint32_t seq0, int n_pre,
                                            Fn&& fn) {
  constexpr int VEC = VecT<T>::N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t S = (uint32_t)sp.stages;
  const uint32_t chunk = (uint32_t)sp.chunk;
  const int n_chunks = (int)((t1 - t0 + chunk - 1) / chunk);
  bool failed = false;
  int issued = n_pre;
  if (warp == kWarps) {
    if (lane == 0) {
      for (int cn = n_pre; cn < n_chunks && !failed; ++cn) {
        const uint32_t q = seq0 + (uint32_t)cn, st = q % S;
        if (!mbar_wait(v.ebar + st, ((q / S) - 1) & 1u, a.err)) {
          failed = true;
          break;
        }
        fence_proxy_async();
        const uint32_t e = t0 + (uint32_t)cn * chunk;
        const uint32_t ne = (min(chunk, t1 - e) + VEC - 1) / VEC * VEC;
        mbar_expect_tx(v.bar + st, ne * (uint32_t)sizeof(T));
        bulk_g2s(v.buf + (size_t)st * chunk, tab + e, ne * (uint32_t)sizeof(T), v.bar + st);
        issued = cn + 1;
      }
    }
  } else {
    for (int ci = 0; ci < n_chunks; ++ci) {
      const uint32_t q = seq0 + (uint32_t)ci, st = q % S;
      if (!mbar_wait(v.bar + st, (q / S) & 1u, a.err)) {
        failed = true;
        break;
      }
      const uint32_t ce = t0 + (uint32_t)ci * chunk;
      fn(ce, min(t1, ce + chunk), v.buf + (size_t)st * chunk);
      __syncwarp();
      if (lane == 0) mbar_arrive(v.ebar + st);  // this warp is done with the stage
    }
  }
  if (__syncthreads_or(failed)) {
    if (warp == kWarps && lane == 0) {
      atomicExch(a.err, 1);
      // the producer runs at most S chunks ahead of the slowest consumer
      for (int cj = max(0, issued - (int)S); cj < issued; ++cj) {
        const uint32_t q = seq0 + (uint32_t)cj;
        mbar_wait(v.bar + q % S, (q / S) & 1u, nullptr);
      }
    }
    return false;
  }
  return true;
}

// Load the consumer thread's kVpt vectors of a staged chunk (zeros past the end).
template <typename T>
__device__ __forceinline__ void load_chunk(const T* sb, uint32_t ce, uint32_t cend, T (&xs)[kVpt][VecT<T>::N]) {
  constexpr int VEC = VecT<T>::N;
  const int nvec = (int)((cend - ce + VEC - 1) / VEC);
#pragma unroll
  for (int it = 0; it < kVpt; ++it) {
    const int i = it * kThreads + (int)threadIdx.x;
    if (i < nvec) {
      VecT<T>::lds(sb + (size_t)i * VEC, xs[it]);
    } else {
#pragma unroll
      for (int j = 0; j < VEC; ++j) xs[it][j] = T(0);
    }
#pragma unroll
    for (int j = 0; j < VEC; ++j)
      if (ce + (uint32_t)i * VEC + j >= cend) xs[it][j] = T(0);
  }
}

// Stream the slice through the bulk-copy ring: per entry v = phi E_col
// (times G for distribute); row sums R(r) = sum_col v; distribute also
// accumulates the column joint and writes the calibrated entry.  Chunks carry
// a per-CTA sequence number `seq0 + ci`, so ring stages and mbarrier phases
// continue across the CTA's items.  The producer warp refills a stage once
// every consumer warp released it; consumer warps never wait for each other.
// Returns false (after letting issued copies land) if a wait timed out.
template <typename T, bool COLLECT, bool POW2, bool ROWVEC, int CBMAX>
__device__ __forceinline__ bool stream(const LevelArgs<T>& a, const SmemPlan& sp, const DevClique& c,
                                       const CtaView<T>& v, const SliceGeo& g, const T* tab, int cb0, int ncb,
                                       uint32_t seq0, int n_pre) {
  constexpr int VEC = VecT<T>::N;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t P = g.P, t0 = g.t0;
  const bool has_joint = c.joint_off >= 0;
  const bool regjoint = !COLLECT && has_joint && ((uint32_t)sp.chunk % P == 0u);
  const bool row_in_warp = POW2 && ROWVEC && P <= 32u * VEC;
  const bool p1 = (P == 1u);
  // column-joint accumulators per vector slot: the columns a thread sees in
  // slot `it` repeat every chunk when P divides the chunk
  T jacc[CBMAX][kVpt][VEC];
#pragma unroll
  for (int cl = 0; cl < CBMAX; ++cl)
#pragma unroll
    for (int it = 0; it < kVpt; ++it)
#pragma unroll
      for (int j = 0; j < VEC; ++j) jacc[cl][it][j] = T(0);
  const bool ok = ring_stream<T>(a, sp, v, tab, g.t0, g.t1, seq0, n_pre, [&](uint32_t ce, uint32_t cend, const T* sb) {
    T xs[kVpt][VEC];
    load_chunk<T>(sb, ce, cend, xs);
    const int nvec = (int)((cend - ce + VEC - 1) / VEC);
#pragma unroll
    for (int it = 0; it < kVpt; ++it) {
      if (it * kThreads + (tid & ~31) >= nvec) break;  // warp-uniform
      const int i = it * kThreads + tid;
      const bool act = i < nvec;
      const uint32_t e0 = ce + (uint32_t)i * VEC;
      const T (&x)[VEC] = xs[it];
      if (ROWVEC) {
        const uint32_t ea = act ? e0 : t0;
        const uint32_t rr = row_of<POW2>(c, ea);
        const uint32_t pr = rr - g.r_lo, col0 = ea - rr * P;
        T outv[CBMAX][VEC];
#pragma unroll
        for (int cl = 0; cl < CBMAX; ++cl) {
          T sum = T(0);
          if (cl < ncb) {
            const T G = COLLECT ? T(1) : v.gsm[(size_t)cl * sp.rowmax + pr];
            const bool cm = v.nobs[sp.cb + cl] != 0;
#pragma unroll
            for (int j = 0; j < VEC; ++j) {
              T o = x[j];
              if (cm) o *= colmask<T, POW2>(v, sp, cl, col0 + j);
              if (!COLLECT) {
                o *= G;
                if (regjoint) jacc[cl][it][j] += o;
                else if (has_joint && o != T(0)) atomicAdd(v.jntp[cl] + col0 + j, o);
              }
              outv[cl][j] = o;
              sum += o;
            }
            T* rs = v.rsum + (size_t)cl * sp.rowmax;
            if (POW2) {
              const uint32_t w = min(P / VEC, 32u);  // lanes sharing the row
              for (uint32_t o = 1; o < w; o <<= 1) sum += __shfl_xor_sync(kFull, sum, o);
              if (act && (lane & (w - 1)) == 0) {
                if (row_in_warp) rs[pr] = sum;
                else atomicAdd(rs + pr, sum);
              }
            } else if (act) {
              atomicAdd(rs + pr, sum);
            }
          }
        }
        if (!COLLECT && a.calib != nullptr && act) {
#pragma unroll
          for (int cl = 0; cl < CBMAX; ++cl)
            if (cl < ncb) VecT<T>::store(a.calib + (int64_t)(cb0 + cl) * a.calib_stride + c.base_off + e0, outv[cl]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
          if (act && e0 + j < cend) {
            const uint32_t e = e0 + j;
            const uint32_t rr = row_of<POW2>(c, e);
            const uint32_t pr = rr - g.r_lo, col = e - rr * P;
#pragma unroll
            for (int cl = 0; cl < CBMAX; ++cl) {
              if (cl < ncb) {
                T o = x[j];
                if (v.nobs[sp.cb + cl]) o *= colmask<T, POW2>(v, sp, cl, col);
                if (!COLLECT) {
                  o *= v.gsm[(size_t)cl * sp.rowmax + pr];
                  if (has_joint && o != T(0)) atomicAdd(v.jntp[cl] + col, o);
                  if (a.calib != nullptr) a.calib[(int64_t)(cb0 + cl) * a.calib_stride + c.base_off + e] = o;
                }
                T* rs = v.rsum + (size_t)cl * sp.rowmax + pr;
                if (p1) *rs = o;
                else atomicAdd(rs, o);
              }
            }
          }
        }
      }
    }
  });
  if (!ok) return false;
  if (regjoint && tid < kThreads) {
#pragma unroll
    for (int it = 0; it < kVpt; ++it) {
      const uint32_t colt = (t0 + (uint32_t)(it * kThreads + tid) * VEC) % P;
#pragma unroll
      for (int cl = 0; cl < CBMAX; ++cl)
        if (cl < ncb)
#pragma unroll
          for (int j = 0; j < VEC; ++j)
            if (jacc[cl][it][j] != T(0)) atomicAdd(v.jntp[cl] + (colt + j) % P, jacc[cl][it][j]);
    }
  }
  return true;
}

// Stream a slice of a power-of-two clique whose rows are short, doing all row
// work inline (no per-slice row buffers):
//   P == 1 (no private variables; the fastest cardinality a multiple of the
//          vector width): the entries of a vector differ only in the fastest
//          digit, so every child key is computed once per vector and stepped
//          by the child's w_last;
//   VEC <= P <= 32 VEC: a vector lies in one row and a row in one warp
//          iteration; each lane computes its row factor (lanes of one row read
//          the same shared-memory words), a segmented shuffle forms the row
//          sum, and the row's first lane adds the row outputs.
template <typename T, bool COLLECT, int CBMAX>
__device__ __forceinline__ bool stream_inline(const LevelArgs<T>& a, const SmemPlan& sp, const DevClique& c,
                                              const CtaView<T>& v, const SliceGeo& g, const T* tab, int cb0,
                                              int ncb, uint32_t seq0, int n_pre, bool is_root, bool out_smem) {
  constexpr int VEC = VecT<T>::N;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t P = g.P;
  const bool p1 = (P == 1u);
  const int nch = c.n_child, klast = c.k - 1;
  const uint32_t w = p1 ? 1u : P / VEC;           // lanes sharing a row
  const bool seg_vec = !p1 || (c.LR % VEC) == 0;  // the vector's entries share the parent entry
  const bool has_joint = c.joint_off >= 0;
  // P divides the chunk (P <= 32 VEC), so each slot's columns repeat every chunk
  T jacc[CBMAX][kVpt][VEC];
#pragma unroll
  for (int cl = 0; cl < CBMAX; ++cl)
#pragma unroll
    for (int it = 0; it < kVpt; ++it)
#pragma unroll
      for (int j = 0; j < VEC; ++j) jacc[cl][it][j] = T(0);
  const bool ok = ring_stream<T>(a, sp, v, tab, g.t0, g.t1, seq0, n_pre, [&](uint32_t ce, uint32_t cend, const T* sb) {
    T xs[kVpt][VEC];
    load_chunk<T>(sb, ce, cend, xs);
    const int nvec = (int)((cend - ce + VEC - 1) / VEC);
#pragma unroll
    for (int it = 0; it < kVpt; ++it) {
      if (it * kThreads + (tid & ~31) >= nvec) break;  // warp-uniform
      const int i = it * kThreads + tid;
      const bool act = i < nvec;
      const uint32_t e0 = act ? ce + (uint32_t)i * VEC : g.t0;
      const uint32_t r = p1 ? e0 : (e0 >> c.logP);    // row (P == 1: of the vector's first entry)
      const uint32_t col0 = e0 - r * P;
      // factor per entry: E_row x prod_g mu_g (x rho for distribute), times phi E_col
      T f[CBMAX][VEC];
#pragma unroll
      for (int cl = 0; cl < CBMAX; ++cl) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) f[cl][j] = act ? xs[it][j] : T(0);
        if (cl < ncb) {
          for (int o = 0; o < v.nobs[cl]; ++o) {
            const int2 ob = v.obs[cl * sp.k + o];
            const uint32_t d0 = digit<true>(r, v.pos[ob.x]);
#pragma unroll
            for (int j = 0; j < VEC; ++j)
              if (((p1 && ob.x == klast) ? d0 + j : d0) != (uint32_t)ob.y) f[cl][j] = T(0);
          }
          if (!p1 && v.nobs[sp.cb + cl]) {
#pragma unroll
            for (int j = 0; j < VEC; ++j) f[cl][j] *= colmask<T, true>(v, sp, cl, col0 + j);
          }
        }
      }
      for (int t = 0; t < nch; ++t) {
        const uint32_t k0 = eval_key<true>(r, v.fld + v.ch[t].field_rel, v.ch[t].n_field);
        const uint32_t wl = p1 ? (uint32_t)v.ch[t].w_last : 0u;
#pragma unroll
        for (int cl = 0; cl < CBMAX; ++cl)
          if (cl < ncb) {
            const T* fp = v.facp[cl * sp.n_child + t];
            if (wl == 0u) {
              const T fv = fp[k0];
#pragma unroll
              for (int j = 0; j < VEC; ++j) f[cl][j] *= fv;
            } else {
#pragma unroll
              for (int j = 0; j < VEC; ++j) f[cl][j] *= fp[k0 + j * wl];
            }
          }
      }
      const uint32_t s0 = r >> c.logLR;
      if (COLLECT) {
#pragma unroll
        for (int cl = 0; cl < CBMAX; ++cl)
          if (cl < ncb) {
            if (seg_vec) {
              T sum = T(0);
#pragma unroll
              for (int j = 0; j < VEC; ++j) sum += f[cl][j];
              add_combined(v.win + (int64_t)cl * sp.win, s0 - g.seg_lo, sum, lane);
            } else {
#pragma unroll
              for (int j = 0; j < VEC; ++j)
                add_combined(v.win + (int64_t)cl * sp.win, ((r + j) >> c.logLR) - g.seg_lo, f[cl][j], lane);
            }
          }
      } else {
        if (!is_root) {
#pragma unroll
          for (int cl = 0; cl < CBMAX; ++cl)
            if (cl < ncb) {
              if (seg_vec) {
                const T rh = v.rhop[cl][s0];
#pragma unroll
                for (int j = 0; j < VEC; ++j) f[cl][j] *= rh;
              } else {
#pragma unroll
                for (int j = 0; j < VEC; ++j) f[cl][j] *= v.rhop[cl][(r + j) >> c.logLR];
              }
            }
        }
        // row sums over the lanes of a row (P > 1) and the row outputs
        T rs[CBMAX];
#pragma unroll
        for (int cl = 0; cl < CBMAX; ++cl) {
          rs[cl] = T(0);
#pragma unroll
          for (int j = 0; j < VEC; ++j) rs[cl] += f[cl][j];
          for (uint32_t o = 1; o < w; o <<= 1) rs[cl] += __shfl_xor_sync(kFull, rs[cl], o);
          if ((lane & (w - 1)) != 0) rs[cl] = T(0);  // the row's first lane adds it
        }
        for (int t = 0; t < nch; ++t) {
          const uint32_t k0 = eval_key<true>(r, v.fld + v.ch[t].field_rel, v.ch[t].n_field);
          const uint32_t wl = p1 ? (uint32_t)v.ch[t].w_last : 0u;
#pragma unroll
          for (int cl = 0; cl < CBMAX; ++cl)
            if (cl < ncb) {
              T* op = v.outp[cl * sp.n_child + t];
              if (wl == 0u) {
                add_combined(op, k0, rs[cl], lane);
              } else {
#pragma unroll
                for (int j = 0; j < VEC; ++j) add_combined(op, k0 + j * wl, f[cl][j], lane);
              }
            }
        }
        for (int h = 0; h < c.n_home; ++h) {
          const DevHome hm = v.hm[h];
          const uint32_t d = digit<true>(r, v.pos[hm.pos]);
#pragma unroll
          for (int cl = 0; cl < CBMAX; ++cl)
            if (cl < ncb) add_combined(v.houtp[cl] + (out_smem ? hm.out_off : hm.moff), d, rs[cl], lane);
        }
        if (has_joint) {
#pragma unroll
          for (int cl = 0; cl < CBMAX; ++cl)
#pragma unroll
            for (int j = 0; j < VEC; ++j) jacc[cl][it][j] += f[cl][j];
        }
        if (a.calib != nullptr && act) {
#pragma unroll
          for (int cl = 0; cl < CBMAX; ++cl)
            if (cl < ncb) VecT<T>::store(a.calib + (int64_t)(cb0 + cl) * a.calib_stride + c.base_off + e0, f[cl]);
        }
      }
    }
  });
  if (!ok) return false;
  if (!COLLECT && has_joint && tid < kThreads) {
#pragma unroll
    for (int it = 0; it < kVpt; ++it) {
      const uint32_t colt = (g.t0 + (uint32_t)(it * kThreads + tid) * VEC) % P;
#pragma unroll
      for (int cl = 0; cl < CBMAX; ++cl)
        if (cl < ncb)
#pragma unroll
          for (int j = 0; j < VEC; ++j)
            if (jacc[cl][it][j] != T(0)) atomicAdd(v.jntp[cl] + colt + j, jacc[cl][it][j]);
    }
  }
  return true;
}

// Rows phase after streaming: collect adds R(r) E_row(r) prod_g mu_g[key_g(r)]
// to the parent window; distribute adds R(r) (already x G) to every child
// separator and row-home marginal.
template <typename T, bool COLLECT, bool POW2, int CBMAX>
__device__ __forceinline__ void rows_out(const SmemPlan& sp, const DevClique& c, const CtaView<T>& v,
                                         const SliceGeo& g, int ncb, bool out_smem) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (warp >= kWarps) return;
  const int nch = c.n_child;
  for (int pb = warp * 32; pb < g.nrow; pb += kThreads) {
    const int pr = pb + lane;
    const bool act = pr < g.nrow;
    const uint32_t r = g.r_lo + (act ? (uint32_t)pr : 0u);
    T val[CBMAX];
#pragma unroll
    for (int cl = 0; cl < CBMAX; ++cl) val[cl] = (cl < ncb && act) ? v.rsum[(size_t)cl * sp.rowmax + pr] : T(0);
    if (COLLECT) {
      T F[CBMAX];
      row_factor<T, POW2, CBMAX>(v, sp, nch, ncb, r, F);
      const uint32_t sg = seg_of<POW2>(c, r);
#pragma unroll
      for (int cl = 0; cl < CBMAX; ++cl)
        if (cl < ncb) add_combined(v.win + (int64_t)cl * sp.win, sg - g.seg_lo, F[cl] * val[cl], lane);
    } else {
      for (int t = 0; t < nch; ++t) {
        const uint32_t key = eval_key<POW2>(r, v.fld + v.ch[t].field_rel, v.ch[t].n_field);
#pragma unroll
        for (int cl = 0; cl < CBMAX; ++cl)
          if (cl < ncb) add_combined(v.outp[cl * sp.n_child + t], key, val[cl], lane);
      }
      for (int h = 0; h < c.n_home; ++h) {
        const DevHome hm = v.hm[h];
        const uint32_t d = digit<POW2>(r, v.pos[hm.pos]);
#pragma unroll
        for (int cl = 0; cl < CBMAX; ++cl)
          if (cl < ncb) add_combined(v.houtp[cl] + (out_smem ? hm.out_off : hm.moff), d, val[cl], lane);
      }
    }
  }
}

// Wait until flags[i] != 0 for every i in the list (thread 0 polls, with the
// CTA-uniform result).  Gives up after the wait limit or once another CTA set
// the error word.
__device__ __forceinline__ bool wait_flags(const int32_t* const* flags, int n, int32_t* err, int* s_flag) {
  if (threadIdx.x == 0) {
    bool ok = true;
    const uint64_t t0 = global_ns();
    for (int i = 0; i < n && ok; ++i) {
      while (ld_acquire(flags[i]) == 0) {
        if (ld_acquire(err) != 0 || global_ns() - t0 > kWaitLimitNs) {
          ok = false;
          break;
        }
        __nanosleep(200);
      }
    }
    if (!ok) atomicExch(err, 1);
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// One work item: a slice of one clique for one block of cases, either pass.
// The dependencies of the item (children's collect messages; for distribute
// also the parent's ratio) are awaited as late as possible: a collect slice
// streams its table before it needs its children.
template <typename T, bool COLLECT, int CBMAX>
__device__ bool process_item(const LevelArgs<T>& a, const SmemPlan& sp, const DevWork& w, int cbk,
                             unsigned char* smem, uint32_t& seq) {
  constexpr int VEC = VecT<T>::N;
  const SmemLayout lay(sp);
  DevChild* s_ch = reinterpret_cast<DevChild*>(smem + lay.off_ch);
  DevField* s_fld = reinterpret_cast<DevField*>(smem + lay.off_fld);
  DevHome* s_hm = reinterpret_cast<DevHome*>(smem + lay.off_hm);
  DevPos* s_pos = reinterpret_cast<DevPos*>(smem + lay.off_pos);
  int2* s_obs = reinterpret_cast<int2*>(smem + lay.off_obs);            // [cb][k] row observations
  int2* s_cobs = s_obs + sp.cb * sp.k;                                  // [cb][k] column observations
  int* s_nobs = reinterpret_cast<int*>(smem + lay.off_nobs);            // [cb] row, then [cb] column counts
  const T** s_facp = reinterpret_cast<const T**>(smem + lay.off_facp);  // [cb][n_child]
  T** s_outp = reinterpret_cast<T**>(smem + lay.off_outp);              // [cb][n_child]
  const T** s_rhop = reinterpret_cast<const T**>(smem + lay.off_rhop);  // [cb]
  T** s_houtp = reinterpret_cast<T**>(smem + lay.off_houtp);            // [cb]
  T** s_jntp = reinterpret_cast<T**>(smem + lay.off_jntp);              // [cb]
  T* s_tabs = reinterpret_cast<T*>(smem + lay.off_tabs);
  T* s_win = reinterpret_cast<T*>(smem + lay.off_win);
  double* s_red = reinterpret_cast<double*>(smem + lay.off_red);
  int* s_flag = reinterpret_cast<int*>(s_red + 72);
  const int32_t** s_deps = reinterpret_cast<const int32_t**>(s_red + 40);  // up to 32 dependency flags per batch
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + lay.off_bar);
  uint64_t* s_ebar = s_bar + sp.stages;
  T* s_rsum = reinterpret_cast<T*>(smem + lay.off_rsum);
  T* s_gsm = reinterpret_cast<T*>(smem + lay.off_gsm);
  T* s_buf = reinterpret_cast<T*>(smem + lay.off_buf);

  const int tid = threadIdx.x;
  const uint32_t t0 = (uint32_t)w.t0, t1 = (uint32_t)w.t1;
  const T* tab = a.base + w.base_off;
  const uint32_t S = (uint32_t)sp.stages, chunk = (uint32_t)sp.chunk;
  const int n_chunks = (int)((t1 - t0 + chunk - 1) / chunk);
  const int n_pre = min((int)S, n_chunks);
  const uint32_t seq0 = seq;
  seq += (uint32_t)n_chunks;
  // start streaming the slice at once: descriptors and dependencies overlap it
  if (tid == 0) {
    for (int ci = 0; ci < n_pre; ++ci) {
      const uint32_t q = seq0 + (uint32_t)ci, st = q % S;
      if (q >= S && !mbar_wait(s_ebar + st, ((q / S) - 1) & 1u, a.err)) break;  // stage of an earlier item
      fence_proxy_async();
      const uint32_t e = t0 + (uint32_t)ci * chunk;
      const uint32_t ne = (min(chunk, t1 - e) + VEC - 1) / VEC * VEC;
      mbar_expect_tx(s_bar + st, ne * (uint32_t)sizeof(T));
      bulk_g2s(s_buf + (size_t)st * chunk, tab + e, ne * (uint32_t)sizeof(T), s_bar + st);
    }
  }
  const int cid = w.clique;
  const DevClique c = a.cl[cid];
  const int cb0 = a.case0 + cbk * sp.cb;
  const int ncb = min(sp.cb, a.case0 + a.n_cases - cb0);
  const int nch = c.n_child, k = c.k;
  const bool is_root = (c.depth == 0);
  const int64_t msg = a.msg_total;
  const int64_t off_down = msg, off_rho = 2 * msg, off_marg = 3 * msg, off_joint = 3 * msg + a.marg_total;
  const bool has_joint = c.joint_off >= 0;
  // per-clique residency in the per-case table region (offsets from the plan)
  const bool fac_smem = c.sm_fac >= 0, rho_smem = c.sm_rho >= 0, out_smem = c.sm_out >= 0;
  const bool jnt_smem = c.sm_jnt >= 0;
  auto region = [&](int cl) { return s_tabs + (int64_t)cl * sp.tabs; };
  auto case_acc = [&](int cl) { return a.acc + (int64_t)(cb0 + cl) * a.acc_stride; };
  auto flag_of = [&](int phase, int clique) { return a.done + ((int64_t)phase * a.n_cliques + clique) * a.max_cases + cbk; };

  // ---- prologue: descriptors, evidence, pointers, zeroed accumulators
  for (int i = tid; i < nch; i += kBlock) s_ch[i] = a.ch[c.child_first + i];
  for (int i = tid; i < c.n_field; i += kBlock) s_fld[i] = a.fld[c.field_first + i];
  for (int i = tid; i < k; i += kBlock) s_pos[i] = a.pos[c.pos_first + i];
  if (!COLLECT)
    for (int i = tid; i < c.n_home; i += kBlock) s_hm[i] = a.hm[c.home_first + i];
  if (tid < 2 * sp.cb) s_nobs[tid] = 0;
  if (tid < ncb) {
    T* acc = case_acc(tid);
    s_rhop[tid] = (is_root || COLLECT) ? nullptr
                  : (rho_smem ? (const T*)(region(tid) + c.sm_rho) : (const T*)(acc + off_rho + c.sep_off));
    s_houtp[tid] = out_smem ? region(tid) + c.sm_out : acc + off_marg;
    s_jntp[tid] = !has_joint ? nullptr : (jnt_smem ? region(tid) + c.sm_jnt : acc + off_joint + c.joint_off);
  }
  for (int i = tid; i < sp.cb * sp.rowmax; i += kBlock) s_rsum[i] = T(0);
  if (COLLECT) {
    for (int i = tid; i < ncb * sp.win; i += kBlock) s_win[i] = T(0);
  } else {
    if (out_smem) {
      const int n_out = c.sm_out_len;
      for (int i = tid; i < ncb * n_out; i += kBlock) region(i / n_out)[c.sm_out + i % n_out] = T(0);
    }
    if (jnt_smem && has_joint)
      for (int i = tid; i < ncb * c.P; i += kBlock) region(i / c.P)[c.sm_jnt + i % c.P] = T(0);
  }
  __syncthreads();
  for (int idx = tid; idx < ncb * k; idx += kBlock) {
    const int cl = idx / k, i = idx - cl * k;
    const DevPos P = s_pos[i];
    const int s = a.ev[(int64_t)(cb0 + cl) * a.n_vars + P.var];
    if (s >= 0) {
      if (s >= P.card) {
        atomicOr(&a.status[cb0 + cl], kStatusBadState);
      } else if (!P.is_col) {
        const int slot = atomicAdd(&s_nobs[cl], 1);
        s_obs[cl * sp.k + slot] = make_int2(i, s);
      } else {
        const int slot = atomicAdd(&s_nobs[sp.cb + cl], 1);
        s_cobs[cl * sp.k + slot] = make_int2(i, s);
      }
    }
  }
  for (int idx = tid; idx < ncb * nch; idx += kBlock) {
    const int cl = idx / nch, t = idx - cl * nch;
    const DevChild ch = s_ch[t];
    T* acc = case_acc(cl);
    s_facp[cl * sp.n_child + t] = fac_smem ? (const T*)(region(cl) + c.sm_fac + ch.fac_off)
                                           : (const T*)(acc + ch.sep_off);
    if (!COLLECT)
      s_outp[cl * sp.n_child + t] = out_smem ? region(cl) + c.sm_out + ch.fac_off : acc + off_down + ch.sep_off;
  }
  __syncthreads();

  // dependencies: the children's collect messages (and, for distribute, the
  // parent's ratio), then the factor tables they finalised
  auto await_inputs = [&]() -> bool {
    for (int b = 0; b < nch + 1; b += 32) {
      int nd = 0;
      if (tid == 0) {
        for (int t = b; t < min(nch, b + 32); ++t) s_deps[nd++] = flag_of(0, s_ch[t].child);
        if (!COLLECT && !is_root && b == 0 && nd < 32) s_deps[nd++] = flag_of(1, a.parent_of[cid]);
        s_flag[1] = nd;
      }
      __syncthreads();
      if (!wait_flags(s_deps, s_flag[1], a.err, s_flag)) return false;
    }
    for (int cl = 0; cl < ncb; ++cl) {
      const T* acc = case_acc(cl);
      if (fac_smem) {
        for (int t = 0; t < nch; ++t) {
          const DevChild ch = s_ch[t];
          T* dst = region(cl) + c.sm_fac + ch.fac_off;
          for (int j = tid; j < ch.sep_size; j += kBlock) dst[j] = __ldcg(acc + ch.sep_off + j);
        }
      }
      if (rho_smem && !COLLECT && !is_root) {
        T* dst = region(cl) + c.sm_rho;
        for (int j = tid; j < c.sep_size; j += kBlock) dst[j] = __ldcg(acc + off_rho + c.sep_off + j);
      }
    }
    __syncthreads();
    return true;
  };

  // ---- the slice
  {
    const CtaView<T> v{s_ch,   s_fld,   s_hm,   s_pos, s_obs, s_cobs, s_nobs,  s_facp, s_outp,
                 s_rhop, s_houtp, s_jntp, s_win, s_buf, s_bar,  s_ebar, s_rsum, s_gsm};
    const bool rowvec = (c.P % VEC) == 0;
    const bool inl = inline_rows(c, VEC);
    bool ok = true;
    if (!COLLECT || inl) ok = await_inputs();
    if (ok && inl) {
      const SliceGeo g = slice_geo<true>(c, t0, t1);
      ok = stream_inline<T, COLLECT, CBMAX>(a, sp, c, v, g, tab, cb0, ncb, seq0, n_pre, is_root, out_smem);
    } else if (ok) {
      if (c.pow2) {
        const SliceGeo g = slice_geo<true>(c, t0, t1);
        if (!COLLECT) {
          rows_factor<T, true, CBMAX>(sp, c, v, g, ncb, is_root);
          __syncthreads();
        }
        ok = rowvec ? stream<T, COLLECT, true, true, CBMAX>(a, sp, c, v, g, tab, cb0, ncb, seq0, n_pre)
                    : stream<T, COLLECT, true, false, CBMAX>(a, sp, c, v, g, tab, cb0, ncb, seq0, n_pre);
        if (ok && COLLECT) ok = await_inputs();
        if (ok) rows_out<T, COLLECT, true, CBMAX>(sp, c, v, g, ncb, out_smem);
      } else {
        const SliceGeo g = slice_geo<false>(c, t0, t1);
        if (!COLLECT) {
          rows_factor<T, false, CBMAX>(sp, c, v, g, ncb, is_root);
          __syncthreads();
        }
        ok = rowvec ? stream<T, COLLECT, false, true, CBMAX>(a, sp, c, v, g, tab, cb0, ncb, seq0, n_pre)
                    : stream<T, COLLECT, false, false, CBMAX>(a, sp, c, v, g, tab, cb0, ncb, seq0, n_pre);
        if (ok && COLLECT) ok = await_inputs();
        if (ok) rows_out<T, COLLECT, false, CBMAX>(sp, c, v, g, ncb, out_smem);
      }
    } else if (tid == 0) {
      // the prefetched chunks of this slice must land before the CTA leaves
      for (int ci = 0; ci < n_pre; ++ci) {
        const uint32_t q = seq0 + (uint32_t)ci;
        mbar_wait(s_bar + q % S, (q / S) & 1u, nullptr);
      }
    }
    if (!ok) return false;  // a wait gave up: the error word is set, results are invalid
  }

  // ---- flush the CTA's partial sums
  __syncthreads();
  if (COLLECT) {
    const uint32_t seg_lo = c.pow2 ? seg_of<true>(c, row_of<true>(c, t0)) : seg_of<false>(c, row_of<false>(c, t0));
    const uint32_t seg_hi =
        c.pow2 ? seg_of<true>(c, row_of<true>(c, t1 - 1)) : seg_of<false>(c, row_of<false>(c, t1 - 1));
    const int nwin = (int)(seg_hi - seg_lo + 1);
    for (int idx = tid; idx < ncb * nwin; idx += kBlock) {
      const int cl = idx / nwin, j = idx - cl * nwin;
      const T val = s_win[(int64_t)cl * sp.win + j];
      if (val != T(0)) atomicAdd(case_acc(cl) + c.sep_off + seg_lo + j, val);
    }
  } else {
    for (int cl = 0; cl < ncb; ++cl) {
      T* acc = case_acc(cl);
      if (out_smem) {
        for (int t = 0; t < nch; ++t) {
          const DevChild ch = s_ch[t];
          for (int j = tid; j < ch.sep_size; j += kBlock) {
            const T val = region(cl)[c.sm_out + ch.fac_off + j];
            if (val != T(0)) atomicAdd(acc + off_down + ch.sep_off + j, val);
          }
        }
        for (int h = 0; h < c.n_home; ++h) {
          const DevHome hm = s_hm[h];
          for (int st = tid; st < hm.card; st += kBlock) {
            const T val = region(cl)[c.sm_out + hm.out_off + st];
            if (val != T(0)) atomicAdd(acc + off_marg + hm.moff + st, val);
          }
        }
      }
      if (jnt_smem && has_joint) {
        for (int j = tid; j < c.P; j += kBlock) {
          const T val = region(cl)[c.sm_jnt + j];
          if (val != T(0)) atomicAdd(acc + off_joint + c.joint_off + j, val);
        }
      }
    }
  }

  // ---- the last CTA of this clique (and case block) finalises its messages
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    int32_t* ctr = a.cnt + ((int64_t)(COLLECT ? 0 : 1) * a.n_cliques + cid) * a.max_cases + cbk;
    const int ticket = atomicAdd(ctr, 1);
    const int last = (ticket == w.ntiles - 1);
    if (last) *ctr = 0;  // ready for the next propagation
    *s_flag = last;
  }
  __syncthreads();
  if (!*s_flag) return true;
  __threadfence();

  if (COLLECT) {
    if (!is_root) {  // the root keeps its raw total for log Z
      for (int cl = 0; cl < ncb; ++cl) {
        T* u = case_acc(cl) + c.sep_off;
        double sm = 0.0;
        for (int j = tid; j < c.sep_size; j += kBlock) sm += (double)__ldcg(u + j);
        const double sigma = block_sum(sm, s_red);
        const T scale = sigma > 0.0 ? (T)((double)c.sep_size / sigma) : T(0);
        for (int j = tid; j < c.sep_size; j += kBlock) u[j] = __ldcg(u + j) * scale;
        if (tid == 0) {
          a.ls[(int64_t)(cb0 + cl) * a.n_cliques + cid] =
              sigma > 0.0 ? log(sigma) - log((double)c.sep_size) : -INFINITY;
          if (!(sigma > 0.0)) atomicOr(&a.status[cb0 + cl], kStatusZero);
        }
      }
    }
  } else {
    // child ratios rho_g = new/old (0/0 := 0)
    for (int cl = 0; cl < ncb; ++cl) {
      T* acc = case_acc(cl);
      for (int t = 0; t < nch; ++t) {
        const DevChild ch = s_ch[t];
        const T* d = acc + off_down + ch.sep_off;
        const T* mu = acc + ch.sep_off;
        double sm = 0.0;
        for (int j = tid; j < ch.sep_size; j += kBlock) sm += (double)__ldcg(d + j);
        const double del = block_sum(sm, s_red);
        const T r0 = del > 0.0 ? (T)((double)ch.sep_size / del) : T(0);
        for (int j = tid; j < ch.sep_size; j += kBlock) {
          const T m = __ldcg(mu + j), dv = __ldcg(d + j);
          acc[off_rho + ch.sep_off + j] = m > T(0) ? dv * r0 / m : T(0);
        }
      }
    }
  }
  // publish: the messages of this clique (this case block) are final
  __threadfence();
  __syncthreads();
  if (tid == 0) st_release(flag_of(COLLECT ? 0 : 1, cid), 1);
  return true;
}

// The whole propagation of a case range in one launch: CTAs take work items
// (clique slices x case blocks, collect items deepest level first, then
// distribute items root first) from a queue.  An item's dependencies are
// always earlier in the queue and held by running CTAs, so the schedule
// always progresses; every wait is bounded.
template <typename T, int CBMAX>
__global__ void __launch_bounds__(kBlock, CBMAX == 1 ? 2 : 1) k_propagate(LevelArgs<T> a, SmemPlan sp) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SmemLayout lay(sp);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + lay.off_bar);
  int* s_item = reinterpret_cast<int*>(reinterpret_cast<double*>(smem + lay.off_red) + 76);
  if (threadIdx.x == 0) {
    for (int i = 0; i < sp.stages; ++i) {
      mbar_init(s_bar + i, 1);                   // full: bulk-copy bytes landed
      mbar_init(s_bar + sp.stages + i, kWarps);  // empty: every consumer warp done
    }
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t seq = 0;  // bulk-copy chunks issued by this CTA so far
  for (;;) {
    if (threadIdx.x == 0) *s_item = (ld_acquire(a.err) != 0) ? a.n_items : atomicAdd(a.queue, 1);
    __syncthreads();
    const int it = *s_item;
    __syncthreads();
    if (it >= a.n_items) break;
    const DevWork w = a.work[it];
    const bool ok = w.collect ? process_item<T, true, CBMAX>(a, sp, w, w.cbk, smem, seq)
                              : process_item<T, false, CBMAX>(a, sp, w, w.cbk, smem, seq);
    if (!ok) break;
    __syncthreads();
  }
}

// Normalised marginals (a warp per variable, binned from the variable's
// source table) and log Z(e) (the last CTA along x), per case (y).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_finalize(FinalArgs<T> a) {
  __shared__ double red[kWarps];
  const int cs = a.case0 + (int)blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* acc = a.acc + (int64_t)cs * a.acc_stride;
  if (blockIdx.x == gridDim.x - 1) {
    double s = 0.0;
    for (int c = 1 + tid; c < a.n_cliques; c += kThreads) s += a.ls[(int64_t)cs * a.n_cliques + c];
    s = warp_sum(s);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (tid == 0) {
      int st = a.status[cs];
      double tot = 0.0;
      for (int i = 0; i < kWarps; ++i) tot += red[i];
      const double R = (double)acc[0];  // the root's raw total (root slot at offset 0)
      if (!(R > 0.0) || (st & kStatusZero)) {
        st |= kStatusZero;
        a.logz_out[cs] = -INFINITY;
      } else {
        a.logz_out[cs] = tot + log(R);
      }
      a.status[cs] = st;
    }
    return;
  }
  const int v = (int)blockIdx.x * kWarps + warp;
  if (v >= a.n_vars) return;
  const VarSrc src = a.vs[v];
  double* out = a.marg_out + (int64_t)cs * a.marg_total + src.moff;
  const T* tab = acc + src.off;
  if (src.kind == 0) {
    double z = 0.0;
    for (int x = lane; x < src.card; x += 32) z += (double)tab[x];
    z = warp_sum(z);
    for (int x = lane; x < src.card; x += 32) out[x] = z > 0.0 ? (double)tab[x] / z : NAN;
    return;
  }
  double z = 0.0;
  for (int j = lane; j < src.size; j += 32) z += (double)tab[j];
  z = warp_sum(z);
  const int per = src.size / src.card;  // entries of one state
  for (int x = 0; x < src.card; ++x) {
    double b = 0.0;
    for (int q = lane; q < per; q += 32) {
      const int hi = q / src.st, lo = q - hi * src.st;
      b += (double)tab[(hi * src.card + x) * src.st + lo];
    }
    b = warp_sum(b);
    if (lane == 0) out[x] = z > 0.0 ? b / z : NAN;
  }
}

template <typename T>
__global__ void k_clique_sum(const T* p, int n, double* out) {
  __shared__ double red[kWarps];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) s += (double)p[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kWarps; ++i) t += red[i];
    *out = t;
  }
}

template <typename T>
__global__ void k_clique_gather(const T* p, CliqueOut co, const double* sum, double* out) {
  const double z = *sum;
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

// Every instance asks for the same shared-memory carveout, so SMs never
// re-partition L1/shared memory between consecutive launches.
template <typename T>
void attr_all(int bytes) {
  cudaFuncSetAttribute(k_propagate<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_propagate<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_propagate<T, 1>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_propagate<T, 8>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
}

}  // namespace

int32_t smem_budget(int device) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return 48 * 1024;
  return v;
}

// Kernel attributes (maximum dynamic shared memory, carveout) are set once per
// process, before the first occupancy query or launch.
template <typename T>
void ensure_attrs() {
  static bool done = false;
  if (!done) {
    int dev = 0;
    cudaGetDevice(&dev);
    attr_all<T>(smem_budget(dev));
    done = true;
  }
}

template <typename T>
cudaError_t launch_propagate(const LevelArgs<T>& a, const SmemPlan& sp, int grid, cudaStream_t s) {
  ensure_attrs<T>();
  const int bytes = SmemLayout(sp).bytes;
  if (sp.cb <= 1) {
    k_propagate<T, 1><<<grid, kBlock, bytes, s>>>(a, sp);
  } else {
    k_propagate<T, 8><<<grid, kBlock, bytes, s>>>(a, sp);
  }
  return cudaGetLastError();
}

int32_t propagate_occupancy(int elem, int cb, int bytes) {
  int n = 0;
  cudaError_t e;
  if (elem == 8) ensure_attrs<double>();
  else ensure_attrs<float>();
  if (elem == 8) {
    e = cb <= 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_propagate<double, 1>, kBlock, bytes)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_propagate<double, 8>, kBlock, bytes);
  } else {
    e = cb <= 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_propagate<float, 1>, kBlock, bytes)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_propagate<float, 8>, kBlock, bytes);
  }
  return e == cudaSuccess ? n : 0;
}

template <typename T>
cudaError_t launch_finalize(const FinalArgs<T>& a, cudaStream_t s) {
  if (a.n_cases <= 0) return cudaSuccess;
  dim3 grid((a.n_vars + kWarps - 1) / kWarps + 1, a.n_cases);
  k_finalize<T><<<grid, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_get_clique(const T* calib_clique, const CliqueOut& co, double* out_dev, double* sum_dev,
                              cudaStream_t s) {
  k_clique_sum<T><<<1, kThreads, 0, s>>>(calib_clique, co.n, sum_dev);
  const int blocks = (int)std::min<int64_t>(1024, (co.n + kThreads - 1) / kThreads);
  k_clique_gather<T><<<blocks, kThreads, 0, s>>>(calib_clique, co, sum_dev, out_dev);
  return cudaGetLastError();
}

template cudaError_t launch_propagate<float>(const LevelArgs<float>&, const SmemPlan&, int, cudaStream_t);
template cudaError_t launch_propagate<double>(const LevelArgs<double>&, const SmemPlan&, int, cudaStream_t);
template cudaError_t launch_finalize<float>(const FinalArgs<float>&, cudaStream_t);
template cudaError_t launch_finalize<double>(const FinalArgs<double>&, cudaStream_t);
template cudaError_t launch_get_clique<float>(const float*, const CliqueOut&, double*, double*, cudaStream_t);
template cudaError_t launch_get_clique<double>(const double*, const CliqueOut&, double*, double*, cudaStream_t);

}  // namespace jt

// Message kernels for Hugin propagation on sm_103a.
//
// One launch processes one tree depth ("level") of one pass for a block of
// evidence cases.  Each CTA owns a contiguous slice [t0, t1) of one clique's
// table and a block of cases, and streams the slice once (vector loads of
// 16 bytes):
//
//   collect   (Algorithm 2, Eq. 2):   psi(x) = phi(x) * E(x) * prod_g mu_g(x_Sg)
//             reduced over the contiguous runs of the parent separator;
//   distribute (Algorithm 3, Eq. 3): psi*(x) = psi(x) * rho(x_S), rho = new/old
//             parent separator with 0/0 := 0, reduced into every child
//             separator and into the marginals of variables held only here;
//             optionally written out (the calibrated clique).
//
// mu_g is the collect message of child g normalised to mean one; E(x) is the
// evidence indicator evaluated on the clique's digits; rho is the ratio of the
// parent's distribute message to the stored collect message.  Separator and
// output indices come from the clique's flat index through digit-run fields
// (see jt_internal.h), never from stored index tables.
#include <cmath>
#include <cstdint>

#include "jt_kernels.h"

namespace jt {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
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
  __device__ static void store(float* p, const float (&x)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  }
};
template <>
struct VecT<double> {
  static constexpr int N = 2;
  __device__ static void load(const double* p, double (&x)[2]) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    x[0] = v.x; x[1] = v.y;
  }
  __device__ static void store(double* p, const double (&x)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
  }
};

// n / d for 32-bit n < 2^31, with m = ceil(2^32 / d): umulhi gives the
// quotient or one more; one compare corrects it.
__device__ __forceinline__ uint32_t udiv(uint32_t n, uint32_t d, uint32_t m) {
  if (d == 1u) return n;
  uint32_t q = __umulhi(n, m);
  if (q * d > n) --q;
  return q;
}

template <bool POW2>
__device__ __forceinline__ uint32_t digit(uint32_t e, const DevPos& p) {
  if (POW2) return (e >> p.sh) & ((1u << p.cbits) - 1u);
  uint32_t q = udiv(e, (uint32_t)p.st, p.st_magic);
  return q - udiv(q, (uint32_t)p.card, p.card_magic) * (uint32_t)p.card;
}

template <bool POW2>
__device__ __forceinline__ uint32_t eval_key(uint32_t e, const DevField* f, int nf) {
  uint32_t key = 0;
  for (int i = 0; i < nf; ++i) {
    uint32_t x;
    if (POW2) {
      x = (e >> f[i].sh) & ((1u << f[i].lbits) - 1u);
    } else {
      uint32_t q = udiv(e, (uint32_t)f[i].st, f[i].st_magic);
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
  uint32_t k0 = __shfl_sync(kFull, key, 0);
  if (__all_sync(kFull, key == k0)) {
    v = warp_sum(v);
    if (lane == 0 && v != T(0)) atomicAdd(tab + k0, v);
  } else if (v != T(0)) {
    atomicAdd(tab + key, v);
  }
}

template <typename T, bool COLLECT, bool POW2, bool VECOK, int CBMAX>
__global__ void __launch_bounds__(kThreads) k_level(LevelArgs<T> a, SmemPlan sp) {
  constexpr int VEC = VecT<T>::N;
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout lay(sp);
  DevChild* s_ch = reinterpret_cast<DevChild*>(smem + lay.off_ch);
  DevField* s_fld = reinterpret_cast<DevField*>(smem + lay.off_fld);
  DevHome* s_hm = reinterpret_cast<DevHome*>(smem + lay.off_hm);
  DevSrc* s_src = reinterpret_cast<DevSrc*>(smem + lay.off_src);
  DevPos* s_pos = reinterpret_cast<DevPos*>(smem + lay.off_pos);
  int2* s_obs = reinterpret_cast<int2*>(smem + lay.off_obs);
  int* s_nobs = reinterpret_cast<int*>(smem + lay.off_nobs);
  T** s_facp = reinterpret_cast<T**>(smem + lay.off_facp);
  T** s_outp = reinterpret_cast<T**>(smem + lay.off_outp);
  T* s_scale = reinterpret_cast<T*>(smem + lay.off_scale);
  T** s_houtp = reinterpret_cast<T**>(smem + lay.off_houtp);
  T* s_rho = reinterpret_cast<T*>(smem + lay.off_rho);
  T* s_fac = reinterpret_cast<T*>(smem + lay.off_fac);
  T* s_out = reinterpret_cast<T*>(smem + lay.off_out);
  T* s_srcacc = reinterpret_cast<T*>(smem + lay.off_srcacc);
  double* s_red = reinterpret_cast<double*>(smem + lay.off_red);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const DevWork w = a.work[blockIdx.x];
  const DevClique c = a.cl[w.clique];
  const int cb0 = a.case0 + (int)blockIdx.y * sp.cb;
  const int ncb = min(sp.cb, a.case0 + a.n_cases - cb0);
  const int nch = c.n_child, k = c.k;
  const bool is_root = (c.depth == 0);

  // ---- descriptors into shared memory
  for (int i = tid; i < nch; i += kThreads) s_ch[i] = a.ch[c.child_first + i];
  for (int i = tid; i < k; i += kThreads) s_pos[i] = a.pos[c.pos_first + i];
  for (int i = tid; i < c.n_home; i += kThreads) s_hm[i] = a.hm[c.home_first + i];
  if (!COLLECT)
    for (int i = tid; i < c.n_src; i += kThreads) s_src[i] = a.src[c.src_first + i];
  if (tid < sp.cb) s_nobs[tid] = 0;
  __syncthreads();
  const int f0 = nch ? s_ch[0].field_first : 0;
  const int nf = nch ? s_ch[nch - 1].field_first + s_ch[nch - 1].n_field - f0 : 0;
  for (int i = tid; i < nf; i += kThreads) s_fld[i] = a.fld[f0 + i];
  if (tid == 0) {
    int off = 0;  // running offset of each child table inside a case's factor/output block
    for (int t = 0; t < nch; ++t) {
      s_ch[t].pad0 = off;
      s_ch[t].field_first -= f0;
      off += s_ch[t].sep_size;
    }
    int hoff = 0;  // home outputs follow the child outputs in smem mode
    for (int h = 0; h < c.n_home; ++h) {
      int loc = sp.out_global ? s_hm[h].moff : off + hoff;
      hoff += s_hm[h].card;
      s_hm[h].var = loc;
    }
    int so = 0;
    for (int i = 0; i < (COLLECT ? 0 : c.n_src); ++i) {
      s_src[i].var = so;
      so += s_src[i].card;
    }
  }
  // evidence: (position, state) of observed variables, per case
  for (int idx = tid; idx < ncb * k; idx += kThreads) {
    const int cl = idx / k, i = idx - cl * k;
    const int s = a.ev[(int64_t)(cb0 + cl) * a.n_vars + a.pos[c.pos_first + i].var];
    if (s >= 0) {
      if (s >= a.pos[c.pos_first + i].card) {
        atomicOr(&a.status[cb0 + cl], kStatusBadState);
      } else {
        const int slot = atomicAdd(&s_nobs[cl], 1);
        s_obs[cl * sp.k + slot] = make_int2(i, s);
      }
    }
  }
  __syncthreads();

  // ---- per-case factor tables (warp per table): copy, sum, scale
  const int n_items = ncb * nch;
  for (int q = warp; q < n_items; q += kWarps) {
    const int cl = q / nch, t = q - cl * nch;
    const DevChild ch = s_ch[t];
    T* accc = a.acc + (int64_t)(cb0 + cl) * a.acc_stride;
    const T* u = accc + ch.sep_off;
    T* dst = sp.fac_global ? const_cast<T*>(u) : s_fac + (int64_t)cl * sp.fac + ch.pad0;
    double sum = 0.0;
    for (int j = lane; j < ch.sep_size; j += 32) {
      const T x = u[j];
      if (!sp.fac_global) dst[j] = x;
      sum += (double)x;
    }
    sum = warp_sum(sum);
    if (lane == 0) {
      s_facp[cl * sp.n_child + t] = dst;
      s_scale[cl * sp.n_child + t] = sum > 0.0 ? (T)((double)ch.sep_size / sum) : T(0);
      if (COLLECT && w.tile == 0) {
        a.ls[(int64_t)(cb0 + cl) * a.n_cliques + ch.child] =
            sum > 0.0 ? log(sum) - log((double)ch.sep_size) : -INFINITY;
        if (!(sum > 0.0)) atomicOr(&a.status[cb0 + cl], kStatusZero);
      }
      T* ob = sp.out_global ? accc + a.msg_total + ch.sep_off : s_out + (int64_t)cl * sp.out + ch.pad0;
      s_outp[cl * sp.n_child + t] = ob;
    }
  }
  // parent ratio sums (distribute, non-root): s_red[2cl] = sigma_c, s_red[2cl+1] = Delta_c
  if (!COLLECT && !is_root) {
    for (int q = warp; q < 2 * ncb; q += kWarps) {
      const int cl = q >> 1;
      const T* accc = a.acc + (int64_t)(cb0 + cl) * a.acc_stride;
      const T* src = accc + (q & 1 ? a.msg_total : 0) + c.sep_off;
      double sum = 0.0;
      for (int j = lane; j < c.sep_size; j += 32) sum += (double)src[j];
      sum = warp_sum(sum);
      if (lane == 0) s_red[q] = sum;
    }
  }
  if (tid < ncb) {
    T* accc = a.acc + (int64_t)(cb0 + tid) * a.acc_stride;
    s_houtp[tid] = sp.out_global ? accc + 2 * (int64_t)a.msg_total : s_out + (int64_t)tid * sp.out;
  }
  // zero shared accumulators
  if (!sp.out_global || COLLECT)
    for (int i = tid; i < ncb * sp.out; i += kThreads) s_out[i] = T(0);
  for (int i = tid; i < ncb * sp.srcacc; i += kThreads) s_srcacc[i] = T(0);
  __syncthreads();

  // ---- parent ratio rho = (new / old) with 0/0 := 0, and separator-read marginals
  if (!COLLECT && !is_root) {
    for (int idx = tid; idx < ncb * c.sep_size; idx += kThreads) {
      const int cl = idx / c.sep_size, j = idx - cl * c.sep_size;
      const T* accc = a.acc + (int64_t)(cb0 + cl) * a.acc_stride;
      const double sig = s_red[2 * cl], del = s_red[2 * cl + 1];
      const T r0 = del > 0.0 ? (T)(sig / del) : T(0);
      const T uo = accc[c.sep_off + j];
      const T dn = accc[a.msg_total + c.sep_off + j];
      s_rho[(int64_t)cl * sp.rho + j] = uo > T(0) ? dn * r0 / uo : T(0);
      if (w.tile == 0) {
        for (int i = 0; i < c.n_src; ++i) {
          const DevSrc sv = s_src[i];
          const int d = (j / sv.st) % sv.card;
          atomicAdd(&s_srcacc[cl * sp.srcacc + sv.var + d], dn);
        }
      }
    }
    __syncthreads();
    if (w.tile == 0) {
      for (int cl = 0; cl < ncb; ++cl) {
        T* marg = a.acc + (int64_t)(cb0 + cl) * a.acc_stride + 2 * (int64_t)a.msg_total;
        for (int i = 0; i < c.n_src; ++i) {
          const DevSrc sv = a.src[c.src_first + i];
          for (int s = tid; s < sv.card; s += kThreads)
            marg[sv.moff + s] = s_srcacc[cl * sp.srcacc + s_src[i].var + s];
        }
      }
    }
  }

  // ---- stream the slice
  const uint32_t t0 = (uint32_t)w.t0, t1 = (uint32_t)w.t1;
  const uint32_t L = (uint32_t)c.L, Lm = c.L_magic;
  const uint32_t seg_lo = udiv(t0, L, Lm);
  const bool seg_vec = (L % VEC) == 0;
  const int nvec = (int)((t1 - t0 + VEC - 1) / VEC);
  const T* tab = a.base + c.base_off;
  for (int vb = warp * 32; vb < nvec; vb += kThreads) {
    const int i = vb + lane;
    const bool act = i < nvec;
    const uint32_t e0 = t0 + (uint32_t)i * VEC;
    T x[VEC];
    if (act) {
      VecT<T>::load(tab + e0, x);
    } else {
#pragma unroll
      for (int j = 0; j < VEC; ++j) x[j] = T(0);
    }
    bool valid[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      valid[j] = act && (e0 + j < t1);
      if (!valid[j]) x[j] = T(0);
    }

    T prod[CBMAX][VEC];
    // evidence indicator
#pragma unroll
    for (int cl = 0; cl < CBMAX; ++cl) {
      bool ok[VEC];
#pragma unroll
      for (int j = 0; j < VEC; ++j) ok[j] = true;
      if (cl < ncb) {
        for (int o = 0; o < s_nobs[cl]; ++o) {
          const int2 ob = s_obs[cl * sp.k + o];
          const DevPos P = s_pos[ob.x];
          if (VECOK) {
            const uint32_t d0 = digit<POW2>(e0, P);
            const bool last = (ob.x == k - 1);
#pragma unroll
            for (int j = 0; j < VEC; ++j) ok[j] = ok[j] && ((last ? d0 + j : d0) == (uint32_t)ob.y);
          } else {
#pragma unroll
            for (int j = 0; j < VEC; ++j) ok[j] = ok[j] && (digit<POW2>(e0 + j, P) == (uint32_t)ob.y);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < VEC; ++j) prod[cl][j] = ok[j] ? x[j] : T(0);
    }
    // child factors mu_g (collect messages, normalised by their scale)
    for (int t = 0; t < nch; ++t) {
      const DevField* F = s_fld + s_ch[t].field_first;
      const int nft = s_ch[t].n_field;
      uint32_t key[VEC];
      if (VECOK) {
        const uint32_t k0 = eval_key<POW2>(e0, F, nft), wl = (uint32_t)s_ch[t].w_last;
#pragma unroll
        for (int j = 0; j < VEC; ++j) key[j] = k0 + j * wl;
      } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) key[j] = eval_key<POW2>(e0 + j, F, nft);
      }
#pragma unroll
      for (int cl = 0; cl < CBMAX; ++cl) {
        if (cl < ncb) {
          const T* fp = s_facp[cl * sp.n_child + t];
          const T sc = s_scale[cl * sp.n_child + t];
#pragma unroll
          for (int j = 0; j < VEC; ++j) prod[cl][j] *= fp[key[j]] * sc;
        }
      }
    }
    uint32_t seg[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) seg[j] = valid[j] ? udiv(e0 + j, L, Lm) : seg_lo;

    if (COLLECT) {
      // Eq. 2 towards the parent: contiguous runs of the parent separator
#pragma unroll
      for (int cl = 0; cl < CBMAX; ++cl) {
        if (cl < ncb) {
          T* outc = s_out + (int64_t)cl * sp.out;
          if (VECOK && seg_vec) {
            T v = T(0);
#pragma unroll
            for (int j = 0; j < VEC; ++j) v += prod[cl][j];
            add_combined(outc, seg[0] - seg_lo, v, lane);
          } else {
#pragma unroll
            for (int j = 0; j < VEC; ++j) add_combined(outc, seg[j] - seg_lo, prod[cl][j], lane);
          }
        }
      }
    } else {
      // Eq. 3: scatter the parent ratio, then reduce into the children and homes
      if (!is_root) {
#pragma unroll
        for (int cl = 0; cl < CBMAX; ++cl)
          if (cl < ncb) {
            const T* r = s_rho + (int64_t)cl * sp.rho;
#pragma unroll
            for (int j = 0; j < VEC; ++j) prod[cl][j] *= r[seg[j]];
          }
      }
      if (a.calib != nullptr && act) {
#pragma unroll
        for (int cl = 0; cl < CBMAX; ++cl)
          if (cl < ncb) VecT<T>::store(a.calib + (int64_t)(cb0 + cl) * a.calib_stride + c.base_off + e0, prod[cl]);
      }
      for (int t = 0; t < nch; ++t) {
        const DevField* F = s_fld + s_ch[t].field_first;
        const int nft = s_ch[t].n_field;
        const uint32_t wl = (uint32_t)s_ch[t].w_last;
        uint32_t key[VEC];
        if (VECOK) {
          const uint32_t k0 = eval_key<POW2>(e0, F, nft);
#pragma unroll
          for (int j = 0; j < VEC; ++j) key[j] = k0 + j * wl;
        } else {
#pragma unroll
          for (int j = 0; j < VEC; ++j) key[j] = eval_key<POW2>(e0 + j, F, nft);
        }
#pragma unroll
        for (int cl = 0; cl < CBMAX; ++cl) {
          if (cl < ncb) {
            T* op = s_outp[cl * sp.n_child + t];
            if (VECOK && wl == 0) {
              T v = T(0);
#pragma unroll
              for (int j = 0; j < VEC; ++j) v += prod[cl][j];
              add_combined(op, key[0], v, lane);
            } else {
#pragma unroll
              for (int j = 0; j < VEC; ++j) add_combined(op, key[j], prod[cl][j], lane);
            }
          }
        }
      }
      for (int h = 0; h < c.n_home; ++h) {
        const DevHome hm = s_hm[h];
        const DevPos P = s_pos[hm.pos];
        const bool last = VECOK && (hm.pos == k - 1);
        uint32_t d[VEC];
        if (VECOK) {
          const uint32_t d0 = digit<POW2>(e0, P);
#pragma unroll
          for (int j = 0; j < VEC; ++j) d[j] = last ? d0 + j : d0;
        } else {
#pragma unroll
          for (int j = 0; j < VEC; ++j) d[j] = valid[j] ? digit<POW2>(e0 + j, P) : 0u;
        }
#pragma unroll
        for (int cl = 0; cl < CBMAX; ++cl) {
          if (cl < ncb) {
            T* op = s_houtp[cl] + hm.var;
            if (VECOK && !last) {
              T v = T(0);
#pragma unroll
              for (int j = 0; j < VEC; ++j) v += prod[cl][j];
              add_combined(op, d[0], v, lane);
            } else {
#pragma unroll
              for (int j = 0; j < VEC; ++j) add_combined(op, d[j], prod[cl][j], lane);
            }
          }
        }
      }
    }
  }
  __syncthreads();

  // ---- flush shared accumulators to the per-case message / marginal arrays
  if (COLLECT) {
    const uint32_t seg_hi = udiv(t1 - 1, L, Lm);
    const int nwin = (int)(seg_hi - seg_lo + 1);
    for (int idx = tid; idx < ncb * nwin; idx += kThreads) {
      const int cl = idx / nwin, j = idx - cl * nwin;
      const T v = s_out[(int64_t)cl * sp.out + j];
      if (v != T(0)) atomicAdd(a.acc + (int64_t)(cb0 + cl) * a.acc_stride + c.sep_off + seg_lo + j, v);
    }
  } else if (!sp.out_global) {
    for (int cl = 0; cl < ncb; ++cl) {
      T* accc = a.acc + (int64_t)(cb0 + cl) * a.acc_stride;
      for (int t = 0; t < nch; ++t) {
        const DevChild ch = s_ch[t];
        for (int j = tid; j < ch.sep_size; j += kThreads) {
          const T v = s_out[(int64_t)cl * sp.out + ch.pad0 + j];
          if (v != T(0)) atomicAdd(accc + a.msg_total + ch.sep_off + j, v);
        }
      }
      for (int h = 0; h < c.n_home; ++h) {
        const DevHome hm = s_hm[h];
        const int moff = a.hm[c.home_first + h].moff;
        for (int s = tid; s < hm.card; s += kThreads) {
          const T v = s_out[(int64_t)cl * sp.out + hm.var + s];
          if (v != T(0)) atomicAdd(accc + 2 * (int64_t)a.msg_total + moff + s, v);
        }
      }
    }
  }
}

// log Z(e) and normalised marginals, one CTA per case.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_finalize(FinalArgs<T> a) {
  __shared__ double red[kWarps];
  const int cs = a.case0 + (int)blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* accc = a.acc + (int64_t)cs * a.acc_stride;
  double s = 0.0;
  for (int c = 1 + tid; c < a.n_cliques; c += kThreads) s += a.ls[(int64_t)cs * a.n_cliques + c];
  s = warp_sum(s);
  if (lane == 0) red[warp] = s;
  __syncthreads();
  int st = a.status[cs];
  if (tid == 0) {
    double tot = 0.0;
    for (int i = 0; i < kWarps; ++i) tot += red[i];
    const double R = (double)accc[a.root_sep_off];
    if (!(R > 0.0) || (st & kStatusZero)) {
      st |= kStatusZero;
      a.logz_out[cs] = -INFINITY;
    } else {
      a.logz_out[cs] = tot + log(R);
    }
    a.status[cs] = st;
  }
  const T* marg = accc + 2 * (int64_t)a.msg_total;
  for (int v = tid; v < a.n_vars; v += kThreads) {
    const int o = a.moff[v], kc = a.card_of[v];
    double z = 0.0;
    for (int x = 0; x < kc; ++x) z += (double)marg[o + x];
    for (int x = 0; x < kc; ++x)
      a.marg_out[(int64_t)cs * a.marg_total + o + x] = z > 0.0 ? (double)marg[o + x] / z : NAN;
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

template <typename T, bool C, bool P, bool V, int CB>
void set_attr(int bytes) {
  cudaFuncSetAttribute(k_level<T, C, P, V, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <typename T, bool C, bool P, bool V>
cudaError_t launch_cb(const LevelArgs<T>& a, const LaunchLevel& L, int bytes, cudaStream_t s) {
  dim3 grid(L.n_work, L.n_caseblk);
  if (L.sp.cb <= 1) {
    k_level<T, C, P, V, 1><<<grid, kThreads, bytes, s>>>(a, L.sp);
  } else {
    k_level<T, C, P, V, 8><<<grid, kThreads, bytes, s>>>(a, L.sp);
  }
  return cudaGetLastError();
}

template <typename T, bool C>
cudaError_t launch_pv(const LevelArgs<T>& a, const LaunchLevel& L, int bytes, cudaStream_t s) {
  if (L.pow2_mode) {
    return L.vec_mode ? launch_cb<T, C, true, true>(a, L, bytes, s) : launch_cb<T, C, true, false>(a, L, bytes, s);
  }
  return L.vec_mode ? launch_cb<T, C, false, true>(a, L, bytes, s) : launch_cb<T, C, false, false>(a, L, bytes, s);
}

template <typename T, bool C>
void attr_all(int bytes) {
  set_attr<T, C, true, true, 1>(bytes);
  set_attr<T, C, true, false, 1>(bytes);
  set_attr<T, C, false, true, 1>(bytes);
  set_attr<T, C, false, false, 1>(bytes);
  set_attr<T, C, true, true, 8>(bytes);
  set_attr<T, C, true, false, 8>(bytes);
  set_attr<T, C, false, true, 8>(bytes);
  set_attr<T, C, false, false, 8>(bytes);
}

}  // namespace

int32_t smem_budget(int device) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return 48 * 1024;
  return v;
}

template <typename T>
cudaError_t launch_level(const LevelArgs<T>& a, const LaunchLevel& L, cudaStream_t s) {
  const int bytes = SmemLayout(L.sp).bytes;
  static bool attr_done = false;  // per dtype instantiation
  if (!attr_done) {
    const int b = smem_budget(0);
    attr_all<T, true>(b);
    attr_all<T, false>(b);
    attr_done = true;
  }
  return L.collect ? launch_pv<T, true>(a, L, bytes, s) : launch_pv<T, false>(a, L, bytes, s);
}

template <typename T>
cudaError_t launch_finalize(const FinalArgs<T>& a, cudaStream_t s) {
  if (a.n_cases <= 0) return cudaSuccess;
  k_finalize<T><<<a.n_cases, kThreads, 0, s>>>(a);
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

template cudaError_t launch_level<float>(const LevelArgs<float>&, const LaunchLevel&, cudaStream_t);
template cudaError_t launch_level<double>(const LevelArgs<double>&, const LaunchLevel&, cudaStream_t);
template cudaError_t launch_finalize<float>(const FinalArgs<float>&, cudaStream_t);
template cudaError_t launch_finalize<double>(const FinalArgs<double>&, cudaStream_t);
template cudaError_t launch_get_clique<float>(const float*, const CliqueOut&, double*, double*, cudaStream_t);
template cudaError_t launch_get_clique<double>(const double*, const CliqueOut&, double*, double*, cudaStream_t);

}  // namespace jt

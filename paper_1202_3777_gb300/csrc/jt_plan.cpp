// Host-side validation and layout planning for a junction tree.
//
// Structure checks follow the definition of a junction tree (Sec. 2.1): a
// tree of cliques (rooted at clique 0), each separator the intersection of two
// adjacent cliques, and the running-intersection property (the cliques that
// hold a variable form a connected subtree).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "jt_internal.h"
#include "jt_kernels.h"

namespace jt {

uint32_t magic_for(uint32_t d) {
  // ceil(2^32 / d); with q = umulhi(n, m) the true quotient is q or q - 1 for
  // every 32-bit n (the kernel corrects with one compare).
  if (d <= 1) return 0;
  return (uint32_t)(((1ull << 32) + d - 1) / d);
}

static bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
static int32_t ilog2(int64_t x) {
  int32_t r = 0;
  while ((1ll << r) < x) ++r;
  return r;
}

#define FAIL(code, msg)      \
  do {                       \
    *err = (msg);            \
    return (code);           \
  } while (0)

jt_status build_plan(const jt_tree_desc* d, Plan* p, std::string* err) {
  if (!d) FAIL(JT_ERR_INVALID_ARG, "null descriptor");
  if (d->n_vars < 1 || d->n_cliques < 1) FAIL(JT_ERR_INVALID_ARG, "need n_vars >= 1 and n_cliques >= 1");
  if (!d->card || !d->clique_off || !d->clique_vars || !d->parent)
    FAIL(JT_ERR_INVALID_ARG, "null array in descriptor");
  if (d->compute != JT_F32 && d->compute != JT_F64) FAIL(JT_ERR_INVALID_ARG, "bad compute dtype");
  if (d->potentials_dtype != JT_F32 && d->potentials_dtype != JT_F64)
    FAIL(JT_ERR_INVALID_ARG, "bad potentials dtype");
  if (d->max_cases < 1) FAIL(JT_ERR_INVALID_ARG, "max_cases must be >= 1");
  if (d->flags & ~JT_MATERIALIZE_CLIQUES) FAIL(JT_ERR_INVALID_ARG, "unknown flag bits");

  const int32_t nv = d->n_vars, nc = d->n_cliques;
  p->n_vars = nv;
  p->n_cliques = nc;
  p->card.assign(d->card, d->card + nv);
  for (int v = 0; v < nv; ++v)
    if (p->card[v] < 2 || p->card[v] > JT_MAX_CARD)
      FAIL(JT_ERR_INVALID_ARG, "variable " + std::to_string(v) + " has cardinality outside [2, 32767]");

  if (d->clique_off[0] != 0) FAIL(JT_ERR_INVALID_ARG, "clique_off[0] must be 0");
  p->vars.resize(nc);
  std::vector<int32_t> seen(nv, -1);
  for (int c = 0; c < nc; ++c) {
    int64_t a = d->clique_off[c], b = d->clique_off[c + 1];
    if (b <= a) FAIL(JT_ERR_INVALID_ARG, "clique " + std::to_string(c) + " is empty");
    if (b - a > JT_MAX_CLIQUE_VARS)
      FAIL(JT_ERR_UNSUPPORTED, "clique " + std::to_string(c) + " has more than 32 variables");
    for (int64_t i = a; i < b; ++i) {
      int32_t v = d->clique_vars[i];
      if (v < 0 || v >= nv) FAIL(JT_ERR_INVALID_ARG, "bad variable id in clique " + std::to_string(c));
      if (seen[v] == c) FAIL(JT_ERR_NOT_A_JUNCTION_TREE, "duplicate variable in clique " + std::to_string(c));
      seen[v] = c;
      p->vars[c].push_back(v);
    }
  }

  // tree rooted at 0
  p->parent.assign(d->parent, d->parent + nc);
  if (p->parent[0] != -1) FAIL(JT_ERR_NOT_A_JUNCTION_TREE, "clique 0 must be the root (parent[0] = -1)");
  for (int c = 1; c < nc; ++c)
    if (p->parent[c] < 0 || p->parent[c] >= nc || p->parent[c] == c)
      FAIL(JT_ERR_NOT_A_JUNCTION_TREE, "bad parent of clique " + std::to_string(c));
  p->depth.assign(nc, -1);
  p->depth[0] = 0;
  std::vector<int32_t> path;
  for (int c = 1; c < nc; ++c) {
    path.clear();
    int x = c;
    while (p->depth[x] < 0) {
      path.push_back(x);
      x = p->parent[x];
      if ((int)path.size() > nc) FAIL(JT_ERR_NOT_A_JUNCTION_TREE, "cycle in parent links");
    }
    int dd = p->depth[x];
    for (int i = (int)path.size() - 1; i >= 0; --i) p->depth[path[i]] = ++dd;
  }
  p->max_depth = *std::max_element(p->depth.begin(), p->depth.end());
  p->children.assign(nc, {});
  for (int c = 1; c < nc; ++c) p->children[p->parent[c]].push_back(c);  // ascending
  p->levels.assign(p->max_depth + 1, {});
  for (int c = 0; c < nc; ++c) p->levels[p->depth[c]].push_back(c);

  // separators and running intersection
  std::vector<int32_t> holders(nv, 0), shared(nv, 0);
  for (int c = 0; c < nc; ++c)
    for (int v : p->vars[c]) holders[v]++;
  p->sep.assign(nc, {});
  std::vector<char> mark(nv, 0);
  for (int c = 1; c < nc; ++c) {
    for (int v : p->vars[p->parent[c]]) mark[v] = 1;
    for (int v : p->vars[c])
      if (mark[v]) p->sep[c].push_back(v);
    for (int v : p->vars[p->parent[c]]) mark[v] = 0;
    std::sort(p->sep[c].begin(), p->sep[c].end());
    for (int v : p->sep[c]) shared[v]++;
  }
  for (int v = 0; v < nv; ++v) {
    if (holders[v] == 0) FAIL(JT_ERR_NOT_A_JUNCTION_TREE, "variable " + std::to_string(v) + " is in no clique");
    if (shared[v] != holders[v] - 1)
      FAIL(JT_ERR_NOT_A_JUNCTION_TREE, "running intersection fails for variable " + std::to_string(v));
  }

  // table sizes and potentials
  p->n_entries.resize(nc);
  p->entries = 0;
  for (int c = 0; c < nc; ++c) {
    int64_t n = 1;
    for (int v : p->vars[c]) {
      n *= p->card[v];
      if (n > JT_MAX_TABLE_ENTRIES)
        FAIL(JT_ERR_UNSUPPORTED, "clique " + std::to_string(c) + " has more than 2^31-16 entries");
    }
    p->n_entries[c] = n;
    p->entries += n;
  }
  for (int64_t i = 0; d->potentials && i < p->entries; ++i) {
    double x = d->potentials_dtype == JT_F64 ? ((const double*)d->potentials)[i]
                                             : (double)((const float*)d->potentials)[i];
    if (!(x >= 0.0) || !std::isfinite(x)) FAIL(JT_ERR_INVALID_ARG, "potentials must be finite and >= 0");
  }
  p->work_per_case = 0;
  for (int c = 1; c < nc; ++c) p->work_per_case += 2 * (p->n_entries[c] + p->n_entries[p->parent[c]]);

  // separator tables: root gets a 1-entry slot (its total), edges follow
  p->sep_size.assign(nc, 1);
  p->sep_off.assign(nc, 0);
  int64_t off = 4;
  for (int c = 1; c < nc; ++c) {
    int64_t s = 1;
    for (int v : p->sep[c]) s *= p->card[v];
    p->sep_size[c] = (int32_t)s;
    p->sep_off[c] = (int32_t)off;
    off += (s + 3) / 4 * 4;  // tables start on 16-byte boundaries (FP32), for bulk copies
    if (off > (1ll << 30)) FAIL(JT_ERR_UNSUPPORTED, "separator tables too large");
  }
  p->msg_total = (int32_t)off;


  // permuted order, top-down (a parent's order is fixed before its children's
  // separators are laid out): the parent separator in the parent's order,
  // then the variables of child separators (most child separators first),
  // then the private variables
  p->pvars.assign(nc, {});
  p->n_private.assign(nc, 0);
  p->pow2.assign(nc, 1);
  std::vector<int32_t> share(nv, 0);
  for (int dd = 0; dd <= p->max_depth; ++dd)
    for (int c : p->levels[dd]) {
      std::vector<int32_t>& pv = p->pvars[c];
      if (c != 0) {
        for (int v : p->sep[c]) mark[v] = 1;
        std::vector<int32_t> s;
        for (int v : p->pvars[p->parent[c]])
          if (mark[v]) s.push_back(v);
        for (int v : p->sep[c]) mark[v] = 0;
        p->sep[c] = s;
      }
      for (int v : p->sep[c]) mark[v] = 1;
      for (int g : p->children[c])
        for (int v : p->sep[g]) share[v]++;
      std::vector<int32_t> rest;
      for (int v : p->vars[c])
        if (!mark[v]) rest.push_back(v);
      std::stable_sort(rest.begin(), rest.end(), [&](int a, int b) {
        if (share[a] != share[b]) return share[a] > share[b];
        return a < b;
      });
      for (int v : rest) p->n_private[c] += share[v] == 0;
      pv = p->sep[c];
      pv.insert(pv.end(), rest.begin(), rest.end());
      for (int v : p->vars[c]) {
        mark[v] = 0;
        share[v] = 0;
        if (!is_pow2(p->card[v])) p->pow2[c] = 0;
      }
    }

  // private joints, both layouts; a layout-1 joint grows from the least
  // significant private position up while it stays within kFineJointEntries
  int64_t jo = 0;
  for (int L = 0; L < 3; ++L) {
    p->joints[L].assign(nc, {});
    for (int c = 0; c < nc; ++c) {
      const int npv = p->n_private[c];
      if (npv == 0) continue;
      const auto& pv = p->pvars[c];
      const int k = (int)pv.size();
      auto add = [&](int lo, int hi, int64_t q) {
        p->joints[L][c].push_back({(int32_t)jo, (int32_t)q, lo, hi - lo});
        jo += (q + 3) / 4 * 4;
      };
      int hi = k;
      int64_t q = 1;
      for (int i = k - 1; i >= k - npv; --i) {
        const int64_t cq = p->card[pv[i]];
        if ((L == 1 && q > 1 && q * cq > kFineJointEntries) || (L == 2 && q > 1)) {
          add(i + 1, hi, q);
          hi = i + 1;
          q = 1;
        }
        q *= cq;
      }
      add(k - npv, hi, q);
      if (jo > (1ll << 30)) FAIL(JT_ERR_UNSUPPORTED, "private-variable joints too large");
    }
  }
  p->joint_total = (int32_t)jo;
  p->msg_stride = (2ll * p->msg_total + p->joint_total + 31) / 32 * 32;

  // marginals: a variable in some separator is binned from the smallest such
  // separator's distribute message; a private variable from its clique's joint
  p->moff.assign(nv, 0);
  int64_t mo = 0;
  for (int v = 0; v < nv; ++v) {
    p->moff[v] = (int32_t)mo;
    mo += p->card[v];
  }
  p->marg_total = (int32_t)mo;
  std::vector<int32_t> src_edge(nv, -1);
  for (int c = 1; c < nc; ++c)
    for (int v : p->sep[c]) {
      const int e = src_edge[v];
      if (e < 0 || p->sep_size[c] < p->sep_size[e]) src_edge[v] = c;
    }
  for (int L = 0; L < 3; ++L) {
    std::vector<VarSrc>& vs = p->vsrc[L];
    vs.assign(nv, VarSrc{});
    for (int v = 0; v < nv; ++v) {
      VarSrc& q = vs[v];
      q.card = p->card[v];
      q.card_out = p->card[v];
      q.moff = p->moff[v];
      const int e = src_edge[v];
      if (e >= 0) {
        q.off = p->msg_total + p->sep_off[e];
        q.size = p->sep_size[e];
        int64_t t = 1;
        for (int i = (int)p->sep[e].size() - 1; i >= 0; --i) {
          if (p->sep[e][i] == v) q.st = (int32_t)t;
          t *= p->card[p->sep[e][i]];
        }
      }
    }
    for (int c = 0; c < nc; ++c) {
      const auto& pv = p->pvars[c];
      for (const Plan::JointGroup& g : p->joints[L][c]) {
        int64_t t = 1;
        for (int i = g.pos0 + g.npos - 1; i >= g.pos0; --i) {
          VarSrc& q = vs[pv[i]];
          q.off = 2 * p->msg_total + g.off;
          q.size = g.size;
          q.st = (int32_t)t;
          t *= p->card[pv[i]];
        }
      }
    }
  }

  // padded offsets (multiples of 32 elements: 128 B for FP32, 256 B for FP64)
  p->base_off.resize(nc);
  int64_t bo = 0;
  for (int c = 0; c < nc; ++c) {
    p->base_off[c] = bo;
    bo += (p->n_entries[c] + 31) / 32 * 32;
  }
  p->base_len = bo;
  return JT_OK;
}

// ---------------------------------------------------------------------------
// Schedule of one propagation shape.
// ---------------------------------------------------------------------------

namespace {

struct PortSpec {
  int32_t kind, tab, size, other, other2;
  std::vector<char> in;   // positions of the clique inside the port's variable set
};

// Fields of a port: maximal runs of consecutive positions inside its
// variable set (the table keeps the clique's order, first most significant).
void port_fields(const std::vector<int64_t>& st, const std::vector<int32_t>& card, const std::vector<char>& in,
                 bool pow2, std::vector<DevField>* out) {
  const int k = (int)in.size();
  int64_t w = 1;
  int i = k - 1;
  while (i >= 0) {
    if (!in[i]) {
      --i;
      continue;
    }
    int j = i;
    int64_t len = card[i];
    while (j - 1 >= 0 && in[j - 1]) {
      --j;
      len *= card[j];
    }
    DevField f{};
    f.st = (int32_t)st[i];
    f.len = (int32_t)len;
    f.st_magic = magic_for((uint32_t)st[i]);
    f.len_magic = magic_for((uint32_t)len);
    f.w = (int32_t)w;
    f.sh = pow2 ? ilog2(st[i]) : 0;
    f.lb = pow2 ? ilog2(len) : 0;
    out->push_back(f);
    w *= len;
    i = j - 1;
  }
}

int64_t eval_key(const std::vector<DevField>& f, int64_t x) {
  int64_t key = 0;
  for (const DevField& q : f) key += ((x / q.st) % q.len) * q.w;
  return key;
}

}  // namespace

jt_status build_schedule(const Plan& p, int elem, int cb, int n_cases, int n_sm, int smem_bytes, Schedule* s,
                         std::string* err, const int8_t* block_shift) {
  for (int q = 0; q < kBlockClasses; ++q) s->block_shift[q] = block_shift ? block_shift[q] : 0;
  const int VEC = 16 / elem;
  const int lv = VEC == 4 ? 2 : 1;
  const int nc = p.n_cliques;
  s->cb = cb;
  s->n_cb = std::max(1, (n_cases + cb - 1) / cb);
  s->chunk = chunk_bytes_for(cb) / elem;
  s->ring = 4;
  s->stages.assign(2 * nc, DevStage{});
  s->ports.clear();
  s->fields.clear();
  s->pos.clear();
  s->deps.clear();
  s->items.clear();
  s->streamed_entries = 0;

  // positions of every clique
  std::vector<int32_t> pos0(nc);
  std::vector<std::vector<int64_t>> stv(nc);
  std::vector<std::vector<int32_t>> cdv(nc);
  s->max_k = 1;
  for (int c = 0; c < nc; ++c) {
    const auto& pv = p.pvars[c];
    const int k = (int)pv.size();
    s->max_k = std::max(s->max_k, k);
    stv[c].assign(k, 1);
    cdv[c].assign(k, 0);
    for (int i = k - 1; i >= 0; --i) {
      cdv[c][i] = p.card[pv[i]];
      if (i + 1 < k) stv[c][i] = stv[c][i + 1] * cdv[c][i + 1];
    }
    pos0[c] = (int32_t)s->pos.size();
    for (int i = 0; i < k; ++i) {
      DevPos q{};
      q.var = pv[i];
      q.card = cdv[c][i];
      q.st = (int32_t)stv[c][i];
      q.st_magic = magic_for((uint32_t)q.st);
      q.card_magic = magic_for((uint32_t)q.card);
      q.sh = p.pow2[c] ? ilog2(stv[c][i]) : 0;
      q.cb = p.pow2[c] ? ilog2(q.card) : 0;
      q.card_ev = p.card_ev.empty() ? q.card : p.card_ev[pv[i]];
      s->pos.push_back(q);
    }
  }

  // entries per (pass, depth), for the block-size target
  std::vector<std::vector<int64_t>> level_n(2, std::vector<int64_t>(p.max_depth + 1, 0));
  for (int c = 0; c < nc; ++c) {
    if (c != 0) level_n[0][p.depth[c]] += p.n_entries[c];
    level_n[1][p.depth[c]] += p.n_entries[c];
  }

  // ports of every stage
  std::vector<std::vector<PortSpec>> specs(2 * nc);
  s->max_ports = 1;
  s->max_fields = 1;
  for (int c = 0; c < nc; ++c) {
    const auto& pv = p.pvars[c];
    const int k = (int)pv.size();
    auto in_of = [&](const std::vector<int32_t>& vs) {
      std::vector<char> in(k, 0);
      for (int v : vs)
        for (int i = 0; i < k; ++i)
          if (pv[i] == v) in[i] = 1;
      return in;
    };
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 0 && c == 0) continue;  // the root's collect total comes from its distribute pass
      auto& sp = specs[pass * nc + c];
      for (int g : p.children[c]) sp.push_back({kPortMu, p.sep_off[g], p.sep_size[g], g, -1, in_of(p.sep[g])});
      if (pass == 1 && c != 0) sp.push_back({kPortRho, p.sep_off[c], p.sep_size[c], c, p.parent[c], in_of(p.sep[c])});
      if (pass == 0) sp.push_back({kPortU, p.sep_off[c], p.sep_size[c], c, -1, in_of(p.sep[c])});
      if (pass == 1) {
        for (int g : p.children[c])
          sp.push_back({kPortDelta, p.msg_total + p.sep_off[g], p.sep_size[g], g, -1, in_of(p.sep[g])});
        for (const Plan::JointGroup& g : p.joints[cb == kCaseLanes ? 2 : (cb > 1 ? 1 : 0)][c]) {
          std::vector<char> in(k, 0);
          for (int i = g.pos0; i < g.pos0 + g.npos; ++i) in[i] = 1;
          sp.push_back({kPortJoint, 2 * p.msg_total + g.off, g.size, c, -1, in});
        }
      }
      s->max_ports = std::max(s->max_ports, (int)sp.size());
      int nf = 0;
      for (const PortSpec& q : sp) {
        std::vector<DevField> f;
        port_fields(stv[c], cdv[c], q.in, p.pow2[c], &f);
        nf += (int)f.size();
      }
      s->max_fields = std::max(s->max_fields, nf);
    }
  }

  // shared memory: what the windows may use once the ring and descriptors fit
  // (the blob bound: every descriptor at its maximum plus the key tables of
  // the most live ports and iterations a fast-path block can have)
  const bool lanes = cb == kCaseLanes;   // case-lane schedule (FP32, power-of-two cliques only)
  if (lanes && elem != 4) {
    *err = "case-lane schedules are FP32 only";
    return JT_ERR_UNSUPPORTED;
  }
  const int max_fast = lanes ? kClMaxPorts : kMaxFastPorts;
  const int blob_bound = desc_bytes(s->max_k, s->max_ports, s->max_fields) +
                         table_bytes(cb, std::min(s->max_ports, max_fast));
  const int fixed = lanes ? SmemLayoutCL(s->ring, s->chunk, blob_bound, 0).bytes
                          : SmemLayout(cb, s->ring, s->chunk, s->max_k, s->max_ports, blob_bound, 0, elem).bytes;
  const int64_t win_budget = (int64_t)(smem_bytes - fixed - 256) / (2ll * cb * elem);  // two buffers
  if (win_budget < (int64_t)s->max_ports * VEC) {
    *err = "the tree's descriptors do not fit in shared memory";
    return JT_ERR_UNSUPPORTED;
  }

  s->win_max = 4;
  for (int pass = 0; pass < 2; ++pass)
    for (int c = 0; c < nc; ++c) {
      DevStage& S = s->stages[pass * nc + c];
      S.clique = c;
      S.pass = pass;
      S.sum_slot = pass * nc + c;
      S.base_off = p.base_off[c];
      S.n = (int32_t)p.n_entries[c];
      S.k = (int32_t)p.pvars[c].size();
      S.pos0 = pos0[c];
      S.port0 = (int32_t)s->ports.size();
      S.field0 = (int32_t)s->fields.size();
      S.dep0 = (int32_t)s->deps.size();
      S.bits = -1;
      if (pass == 0 && c == 0) continue;  // empty stage
      const auto& sp = specs[pass * nc + c];
      const int k = S.k;
      const bool pow2 = p.pow2[c] != 0;
      std::vector<std::vector<DevField>> pf(sp.size());
      for (size_t i = 0; i < sp.size(); ++i) port_fields(stv[c], cdv[c], sp[i].in, pow2, &pf[i]);
      // window entries of every port for a block of the lowest `inb` bits (power of
      // two) or the lowest `inb` positions (generic)
      auto windows = [&](int inb, bool bitwise, std::vector<int64_t>* K) {
        int64_t tot = 0;
        K->assign(sp.size(), 1);
        for (size_t q = 0; q < sp.size(); ++q) {
          int64_t kk = 1;
          for (int i = 0; i < k; ++i) {
            if (!sp[q].in[i]) continue;
            if (bitwise) {
              const int sh = ilog2(stv[c][i]), cbits = ilog2(cdv[c][i]);
              const int inside = std::max(0, std::min(cbits, inb - sh));
              kk <<= inside;
            } else if (i >= k - inb) {
              kk *= cdv[c][i];
            }
          }
          (*K)[q] = kk;
          if (kk > 1) tot += (kk + 3) / 4 * 4;
        }
        return tot;
      };
      int64_t spread = std::max<int64_t>(4096, level_n[pass][p.depth[c]] * s->n_cb / (2ll * ctas_per_sm_for(cb) * n_sm));
      const int shift = s->block_shift[block_class(S.n)];
      spread = shift >= 0 ? spread << shift : std::max<int64_t>(32, spread >> -shift);
      const int64_t target =
          std::min<int64_t>(std::min<int64_t>(1 << 16, (int64_t)kMaxIter * consumers_for(cb) * VEC), spread);
      std::vector<int64_t> K;
      int64_t B = 1;
      // a case-lane block holds at least one tile (32 entries) per warp slice
      const int min_bits = lanes ? 5 : lv;
      if (lanes && !(pow2 && S.n >= 32 && (int)sp.size() <= kClMaxPorts)) {
        *err = "case-lane schedules need power-of-two cliques of at least 32 entries and at most " +
               std::to_string(kClMaxPorts) + " ports";
        return JT_ERR_UNSUPPORTED;
      }
      if (pow2 && S.n >= VEC && (int)sp.size() <= max_fast) {
        const int nbits = ilog2(S.n);
        int bits = min_bits;
        for (int b = nbits; b >= min_bits; --b) {
          if ((1ll << b) > target && b > min_bits) continue;
          if (windows(b, true, &K) <= win_budget) {
            bits = b;
            break;
          }
        }
        windows(bits, true, &K);
        B = 1ll << bits;
        S.bits = bits;
        S.kin = -1;
      } else {
        int kin = 0;
        for (int q = k; q >= 0; --q) {
          int64_t b = 1;
          for (int i = k - q; i < k; ++i) b *= cdv[c][i];
          if (b > target && q > 0) continue;
          if (windows(q, false, &K) <= win_budget) {
            kin = q;
            break;
          }
        }
        windows(kin, false, &K);
        for (int i = k - kin; i < k; ++i) B *= cdv[c][i];
        S.kin = kin;
      }
      S.B = (int32_t)B;
      S.n_blocks = (int32_t)(S.n / B);
      int32_t win = 0, nin = 0;
      for (size_t q = 0; q < sp.size(); ++q) {
        DevPort P{};
        P.kind = sp[q].kind;
        P.tab = sp[q].tab;
        P.size = sp[q].size;
        P.K = (int32_t)K[q];
        P.win = -1;
        if (P.K > 1) {
          P.win = win;
          win += (P.K + 3) / 4 * 4;  // windows start on 16-byte boundaries
        }
        P.other = sp[q].other;
        P.other2 = sp[q].other2;
        P.nf = (int32_t)pf[q].size();
        P.f0 = (int32_t)s->fields.size() - S.field0;
        for (const DevField& f : pf[q]) s->fields.push_back(f);
        if (S.bits >= 0) {
          // lane bits (entry bits lv..lv+4) the key ignores
          uint32_t lf = 0;
          for (int L = 0; L < 5; ++L) {
            const int eb = lv + L;
            bool dep = false;
            if (eb < S.bits)
              for (int i = 0; i < k; ++i)
                if (sp[q].in[i] && eb >= ilog2(stv[c][i]) && eb < ilog2(stv[c][i]) + ilog2(cdv[c][i])) dep = true;
            if (!dep) lf |= 1u << L;
          }
          P.lane_free = lf;
          bool any = false, seq = true;
          for (int j = 0; j < VEC; ++j) {
            P.dvec[j] = (int32_t)eval_key(pf[q], j);
            any = any || P.dvec[j] != 0;
            seq = seq && P.dvec[j] == j;
          }
          P.vmode = !any ? 0 : (seq ? 1 : 2);
          // an output window with as many entries as the block: the key map
          // is one-to-one, so the consumers store instead of accumulating
          if (P.kind != kPortMu && P.kind != kPortRho && P.vmode == 1 && (int64_t)P.K == B) P.vmode |= kVmodeStore;
          // iteration bits: entry bits from log2(consumers * VEC) up to the
          // block's bits; chunk bits: from log2(chunk) up
          const int ib = ilog2((int64_t)consumers_for(cb) * VEC), cbit = ilog2((int64_t)s->chunk);
          P.iter_dep = 0;
          for (int i = 0; i < k; ++i) {
            if (!sp[q].in[i]) continue;
            const int lo = ilog2(stv[c][i]), hi = lo + ilog2(cdv[c][i]);
            if (hi > ib && lo < S.bits) P.iter_dep |= 1;
            if (hi > cbit && lo < S.bits) P.iter_dep |= 2;
            if (hi > ib && lo < std::min(cbit, S.bits)) P.iter_dep |= 4;
          }
        }
        if (P.kind == kPortMu || P.kind == kPortRho) ++nin;
        s->ports.push_back(P);
      }
      S.covered = 0;
      for (int q = 0; q < nin; ++q)
        for (int i = 0; i < k; ++i)
          if (sp[q].in[i]) S.covered |= 1u << i;
      // digits of a padded plan above the tile, those with the largest share
      // of added states first
      S.holes[0] = S.holes[1] = S.holes[2] = 0u;
      if (!p.card_ev.empty() && pow2) {
        std::vector<std::pair<double, uint32_t>> hd;
        for (int i = 0; i < k; ++i) {
          const int32_t ce = p.card_ev[p.pvars[c][i]];
          const int sh = ilog2(stv[c][i]), nb = ilog2(cdv[c][i]);
          if (ce < cdv[c][i] && sh >= 5)
            hd.push_back({(double)ce / cdv[c][i], (uint32_t)sh | (uint32_t)nb << 5 | (uint32_t)ce << 10});
        }
        std::stable_sort(hd.begin(), hd.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
        for (size_t j = 0; j < hd.size() && j < 3; ++j) S.holes[j] = hd[j].second;
      }
      S.np = (int32_t)sp.size();
      S.nin = nin;
      S.nf = (int32_t)s->fields.size() - S.field0;
      S.win_len = win;
      s->win_max = std::max(s->win_max, win);
      s->streamed_entries += S.n;
    }
  // dependencies need every stage's block count, so they come after the blocks
  for (int pass = 0; pass < 2; ++pass)
    for (int c = 0; c < nc; ++c) {
      DevStage& S = s->stages[pass * nc + c];
      S.dep0 = (int32_t)s->deps.size();
      S.ndep = 0;
      if (pass == 0 && c == 0) continue;
      auto dep = [&](int stage) {
        s->deps.push_back(stage);
        s->deps.push_back(s->stages[stage].n_blocks);
        ++S.ndep;
      };
      if (pass == 0 || c == 0) {
        for (int g : p.children[c]) dep(g);            // collect of every child
      } else {
        dep(nc + p.parent[c]);                          // distribute of the parent
      }
    }

  // descriptor blobs: one contiguous copy per stage of everything a work
  // item reads about its stage (one bulk copy fetches it)
  std::vector<int32_t> blob_at(2 * nc, 0), blob_len(2 * nc, 0);
  s->blobs.clear();
  s->blob_max = 16;
  const int NT = consumers_for(cb);
  for (int st = 0; st < 2 * nc; ++st) {
    DevStage& S = s->stages[st];
    if (S.n_blocks == 0) continue;
    // fast path: the ports with windows (inputs first, port order) and their
    // key tables: kt[port][tid] = key(tid * VEC) + window start (16-bit),
    // kiter[port][m] = key(m * consumers * VEC), from the block's own bits
    std::vector<LivePort> live;
    std::vector<int32_t> kit;
    std::vector<uint16_t> ktab;
    S.n_live = S.n_in_live = S.n_iter = 0;
    S.live_off = 0;
    if (S.bits >= 0) {
      const int64_t per_it = (int64_t)NT * VEC;
      S.n_iter = (int32_t)((S.B + per_it - 1) / per_it);
      for (int pi = 0; pi < S.np; ++pi) {
        const DevPort& P = s->ports[S.port0 + pi];
        if (P.K <= 1) continue;
        LivePort L{};
        L.mode = (P.vmode & 3) | ((P.iter_dep & 1) ? kModeIter : 0) | ((P.iter_dep & 2) ? kModeChunk : 0) |
                 ((P.iter_dep & 4) ? kModeInChunk : 0) | ((P.vmode & kVmodeStore) ? kModeStore : 0) |
                 (int32_t)((P.lane_free & 31u) << 3);
        L.port = pi;
        L.win = P.win;
        for (int j = 0; j < 4; ++j) L.dvec[j] = P.dvec[j];
        live.push_back(L);
        if (pi < S.nin) ++S.n_in_live;
      }
      S.n_live = (int32_t)live.size();
    }
    if (S.bits >= 0 && cb == 1) {  // one-case schedules carry the tables in the blob
      const int64_t per_it = (int64_t)NT * VEC;
      if (S.n_iter > kMaxIter) {
        *err = "block longer than the iteration table";
        return JT_ERR_UNSUPPORTED;
      }
      kit.assign((size_t)S.n_live * kMaxIter, 0);
      ktab.assign((size_t)S.n_live * NT, 0);
      const uint32_t bmask = (uint32_t)S.B - 1u;
      for (int li = 0; li < S.n_live; ++li) {
        const DevPort& P = s->ports[S.port0 + live[li].port];
        const DevField* f = &s->fields[S.field0 + P.f0];
        auto key = [&](uint32_t x) {
          uint32_t k = 0;
          for (int q = 0; q < P.nf; ++q) k += ((x >> f[q].sh) & ((1u << f[q].lb) - 1u)) * (uint32_t)f[q].w;
          return k;
        };
        for (int m = 0; m < kMaxIter; ++m)
          kit[(size_t)li * kMaxIter + m] = (int32_t)key((uint32_t)(std::min(m, S.n_iter - 1) * per_it));
        for (int t = 0; t < NT; ++t) {
          // (a thread past the block's end gets a key inside the window)
          const uint32_t v = key(((uint32_t)t * VEC) & bmask) + (uint32_t)P.win;
          if (v > 0xFFFFu) {
            *err = "window keys exceed 16 bits";
            return JT_ERR_UNSUPPORTED;
          }
          ktab[(size_t)li * NT + t] = (uint16_t)v;
        }
      }
      S.live_off = desc_bytes(S.k, S.np, S.nf);
    }
    // case-lane schedules: per port the class of its key over a tile of 32
    // entries and the key tables of the parts of a block offset (CLPort)
    std::vector<CLPort> clp;
    if (S.bits >= 0 && cb == kCaseLanes) {
      const int CH = s->chunk;
      if ((S.B + CH - 1) / CH > kClMaxChunks) {
        *err = "case-lane block longer than the chunk table";
        return JT_ERR_UNSUPPORTED;
      }
      int n_reg = 0;
      for (int li = 0; li < S.n_live; ++li) {
        const DevPort& P = s->ports[S.port0 + live[li].port];
        const DevField* f = &s->fields[S.field0 + P.f0];
        auto key = [&](uint32_t x) {
          uint32_t k = 0;
          for (int q = 0; q < P.nf; ++q) k += ((x >> f[q].sh) & ((1u << f[q].lb) - 1u)) * (uint32_t)f[q].w;
          return k;
        };
        CLPort C{};
        const bool edep = key(1) != 0 || key(2) != 0;
        const bool vdep = key(4) != 0 || key(8) != 0 || key(16) != 0;
        bool ident = edep;
        for (uint32_t x = 1; ident && x < 32u; x <<= 1) ident = key(x) == x;
        C.cls = (live[li].port < S.nin ? kClInput : 0) | (edep ? kClEntry : (vdep ? kClVector : kClTile)) |
                (ident ? kClIdent : 0);
        C.dep = 0;
        for (int b = 0; b < 5; ++b)
          if (key(1u << b) != 0) C.dep |= 1 << b;
        // an output whose key depends only on entry bits 0-1 (a joint over
        // the lowest digit): four sums per tile, the same rows in every tile
        bool tile_only = true;
        for (int b = 5; b < S.bits; ++b) tile_only = tile_only && key(1u << b) == 0;
        const int vf = (~C.dep >> 2) & 7;
        const bool regable = live[li].port >= S.nin && tile_only && !ident &&
                             edep && vf == 7;
        if (regable && n_reg < kClRegSlots) C.cls |= (++n_reg) << kClRegShift;
        for (int j = 0; j < 4; ++j) C.dvec[j] = (int32_t)(key((uint32_t)j) * kClRow);
        for (int v = 0; v < 8; ++v) C.kvec[v] = (int32_t)(key(4u * (uint32_t)v) * kClRow);
        for (int q = 0; q < 16 * kClTiles; ++q) C.kslot[q] = (int32_t)(key((uint32_t)(32 * q)) * kClRow);
        for (int ci = 0; ci < kClMaxChunks; ++ci)
          C.kchunk[ci] = (int32_t)((uint32_t)P.win * kClRow + key((uint32_t)(ci * CH)) * kClRow);
        clp.push_back(C);
      }
      S.live_off = desc_bytes(S.k, S.np, S.nf);
    }
    blob_at[st] = (int32_t)s->blobs.size();
    auto put = [&](const void* src, size_t bytes) {
      const unsigned char* q = static_cast<const unsigned char*>(src);
      for (size_t i = 0; i < bytes; i += sizeof(uint4)) {
        uint4 u{};
        std::memcpy(&u, q + i, std::min(sizeof(uint4), bytes - i));
        s->blobs.push_back(u);
      }
    };
    put(&S, sizeof(DevStage));
    if (S.np) put(&s->ports[S.port0], S.np * sizeof(DevPort));
    if (S.nf) put(&s->fields[S.field0], S.nf * sizeof(DevField));
    put(&s->pos[S.pos0], S.k * sizeof(DevPos));
    if (!clp.empty()) put(clp.data(), clp.size() * sizeof(CLPort));
    if (S.n_live && cb == 1) {
      put(live.data(), live.size() * sizeof(LivePort));
      put(kit.data(), kit.size() * sizeof(int32_t));     // padded to 16 bytes
      put(ktab.data(), ktab.size() * sizeof(uint16_t));
    }
    blob_len[st] = (int32_t)((s->blobs.size() - blob_at[st]) * sizeof(uint4));
    if (S.n_live && (cb == 1 || cb == kCaseLanes) && blob_len[st] != S.live_off + table_bytes(cb, S.n_live)) {
      *err = "stage blob layout mismatch";
      return JT_ERR_UNSUPPORTED;
    }
    s->blob_max = std::max(s->blob_max, blob_len[st]);
  }

  // work items: collect deepest level first, then distribute from the root,
  // one case block at a time and skewed across case blocks: the steps of
  // the sweep (collect levels max_depth..1, then distribute levels
  // 0..max_depth) of case block q come at wave step + q, so while one case
  // block waits for a level to finish, the next one's previous level fills
  // the queue.  Every item's dependencies (same case block, an earlier step)
  // come earlier in the list.
  auto add = [&](int stage, int q) {
    const DevStage& S = s->stages[stage];
    for (int b = 0; b < S.n_blocks; ++b) {
      DevItem it{};
      it.off = S.base_off + (int64_t)b * S.B;
      it.n = S.B;
      it.stage = stage;
      it.block = b;
      it.cbk = q;
      it.blob = blob_at[stage];
      it.blob_bytes = blob_len[stage];
      s->items.push_back(it);
    }
  };
  // Order inside a level, so that the items whose dependencies finish first
  // come first: a collect stage by the queue position of its last child (a
  // clique without children first), a distribute stage by its parent's
  // position, the deeper subtree first among siblings.
  std::vector<int32_t> height(nc, 0);
  for (int dd = p.max_depth; dd >= 1; --dd)
    for (int c : p.levels[dd]) height[p.parent[c]] = std::max(height[p.parent[c]], height[c] + 1);
  std::vector<std::vector<int32_t>> corder(p.max_depth + 1), dorder(p.max_depth + 1);
  std::vector<int32_t> qpos(nc, 0);
  corder[p.max_depth] = p.levels[p.max_depth];
  for (size_t i = 0; i < corder[p.max_depth].size(); ++i) qpos[corder[p.max_depth][i]] = (int32_t)i;
  for (int dd = p.max_depth - 1; dd >= 1; --dd) {
    std::vector<std::pair<int64_t, int32_t>> key;
    for (int c : p.levels[dd]) {
      int64_t k = -1;
      for (int g : p.children[c]) k = std::max<int64_t>(k, qpos[g]);
      key.push_back({k, c});
    }
    std::stable_sort(key.begin(), key.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    for (size_t i = 0; i < key.size(); ++i) {
      corder[dd].push_back(key[i].second);
      qpos[key[i].second] = (int32_t)i;
    }
  }
  dorder[0] = p.levels[0];
  for (size_t i = 0; i < dorder[0].size(); ++i) qpos[dorder[0][i]] = (int32_t)i;
  for (int dd = 1; dd <= p.max_depth; ++dd) {
    std::vector<std::pair<int64_t, int32_t>> key;
    for (int c : p.levels[dd]) key.push_back({(int64_t)qpos[p.parent[c]] * (nc + 1) + (nc - height[c]), c});
    std::stable_sort(key.begin(), key.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    for (size_t i = 0; i < key.size(); ++i) {
      dorder[dd].push_back(key[i].second);
      qpos[key[i].second] = (int32_t)i;
    }
  }
  const int n_steps = 2 * p.max_depth + 1;
  auto step_stages = [&](int step, std::vector<int>& out) {
    out.clear();
    if (step < p.max_depth) {
      for (int c : corder[p.max_depth - step]) out.push_back(c);
    } else {
      for (int c : dorder[step - p.max_depth]) out.push_back(nc + c);
    }
  };
  std::vector<int> st_list;
  for (int wave = 0; wave < n_steps + s->n_cb - 1; ++wave)
    for (int q = 0; q < s->n_cb; ++q) {
      const int step = wave - q;
      if (step < 0 || step >= n_steps) continue;
      step_stages(step, st_list);
      for (int stage : st_list) add(stage, q);
    }
  if (prop_smem_bytes(*s, elem) > smem_bytes) {
    *err = "propagation plan exceeds shared memory";
    return JT_ERR_UNSUPPORTED;
  }
  return JT_OK;
}

int32_t small_smem_bytes(int64_t msg_stride, int32_t msg_total, int32_t n_cliques, int32_t n_vars, int elem,
                         int32_t lv_blob_max) {
  // messages and ratios (element type), then stage totals and scales (FP64),
  // then the case's evidence row (int16), then one level's descriptors, as
  // the whole-tree kernel carves it
  const int64_t b = (((msg_stride + msg_total) * elem + 15) & ~int64_t(15)) + ((24ll * n_cliques + 15) & ~int64_t(15)) +
                    ((2ll * n_vars + 15) & ~int64_t(15)) + 16ll * lv_blob_max;
  return (int32_t)std::min<int64_t>(b + 16, INT32_MAX);
}

jt_status build_small_schedule(const Plan& p, int elem, int n_cases, int n_sm, int smem_bytes, Schedule* s,
                               std::string* err) {
  // one CTA streams every entry of the tree per case: worth it for trees of
  // up to a few hundred thousand entries (beyond, the persistent schedules
  // spread one case over many SMs)
  constexpr int64_t kSmallMaxEntries = 1 << 17;
  if (p.entries > kSmallMaxEntries) {
    *err = "tree too large for one CTA per case";
    return JT_ERR_UNSUPPORTED;
  }
  jt_status st = build_schedule(p, elem, 1, 1, n_sm, smem_bytes, s, err);
  if (st != JT_OK) return st;
  const int nc = p.n_cliques;
  s->cb = kWholeTree;
  s->n_cb = 1;
  Schedule::SmallPlan& sp = s->small;
  sp = Schedule::SmallPlan{};
  sp.stage_blob.assign(2 * nc, -1);
  // each stage's compact descriptors (no per-thread key tables), laid out
  // level by level so that one copy brings a level's into shared memory
  auto put = [&](const void* src, size_t bytes) {
    const unsigned char* q = static_cast<const unsigned char*>(src);
    for (size_t i = 0; i < bytes; i += sizeof(uint4)) {
      uint4 u{};
      std::memcpy(&u, q + i, std::min(sizeof(uint4), bytes - i));
      sp.blobs.push_back(u);
    }
  };
  // a level whose descriptors exceed the staging budget runs as several
  // consecutive groups (its stages are independent of one another)
  constexpr int32_t kStageUnits = 32768 / 16;
  auto level = [&](const std::vector<int32_t>& stages) {
    int32_t l0 = (int32_t)sp.blobs.size();
    auto close = [&]() {
      sp.lv_blob_max = std::max<int32_t>(sp.lv_blob_max, (int32_t)sp.blobs.size() - l0);
      sp.lv_blob_off.push_back((int32_t)sp.blobs.size());
      sp.seg_lv.push_back((int32_t)sp.segs.size());
      sp.lv_stage_off.push_back((int32_t)sp.lv_stage.size());
      ++sp.levels;
      l0 = (int32_t)sp.blobs.size();
    };
    for (int stg : stages) {
      const DevStage& S = s->stages[stg];
      if (S.n_blocks == 0) continue;
      const int32_t units = (desc_bytes(S.k, S.np, S.nf) + 15) / 16;
      if ((int32_t)sp.blobs.size() - l0 + units > kStageUnits && (int32_t)sp.blobs.size() > l0) close();
      sp.lv_stage.push_back(stg);
      sp.stage_blob[stg] = (int32_t)sp.blobs.size() - l0;
      DevStage C = S;
      C.live_off = 0;
      C.n_live = C.n_in_live = 0;
      put(&C, sizeof(DevStage));
      if (S.np) put(&s->ports[S.port0], S.np * sizeof(DevPort));
      if (S.nf) put(&s->fields[S.field0], S.nf * sizeof(DevField));
      put(&s->pos[S.pos0], S.k * sizeof(DevPos));
      for (int e = 0; e < S.n; e += kSmallSeg) sp.segs.push_back(int2{stg, e});
    }
    close();
  };
  sp.lv_blob_off.push_back(0);
  sp.seg_lv.push_back(0);
  sp.lv_stage_off.push_back(0);
  for (int d = p.max_depth; d >= 1; --d) level(p.levels[d]);          // collect: deepest level first
  for (int d = 0; d <= p.max_depth; ++d) {                           // distribute: from the root
    std::vector<int32_t> v;
    for (int c : p.levels[d]) v.push_back(nc + c);
    level(v);
  }
  const int32_t need = small_smem_bytes(p.msg_stride, p.msg_total, p.n_cliques, p.n_vars, elem, sp.lv_blob_max);
  if (need > smem_bytes) {
    *err = "a case's messages and a level's descriptors do not fit one CTA's shared memory";
    return JT_ERR_UNSUPPORTED;
  }
  sp.smem = need;
  // the packed index arrays
  auto put_idx = [&](const std::vector<int32_t>& v) {
    const int32_t o = (int32_t)sp.idx.size();
    sp.idx.insert(sp.idx.end(), v.begin(), v.end());
    if (sp.idx.size() & 1) sp.idx.push_back(0);
    return o;
  };
  sp.idx.clear();
  put_idx(sp.lv_blob_off);
  sp.o_seg_lv = put_idx(sp.seg_lv);
  sp.o_lv_stage_off = put_idx(sp.lv_stage_off);
  sp.o_stage_blob = put_idx(sp.stage_blob);
  sp.o_lv_stage = put_idx(sp.lv_stage);
  sp.o_sep_size = put_idx(p.sep_size);
  sp.o_segs = (int32_t)sp.idx.size();
  for (const int2& g : sp.segs) {
    sp.idx.push_back(g.x);
    sp.idx.push_back(g.y);
  }
  while (sp.idx.size() % 4) sp.idx.push_back(0);
  // what else fits in shared memory, in order of use per entry: the clique
  // tables (read by every entry), the packed indices (per segment), every
  // level's descriptors at once (staged once per CTA instead of once per
  // level and case)
  int64_t used = need;
  if (used + p.base_len * elem <= smem_bytes) {
    sp.base_in_smem = true;
    used += p.base_len * elem;
  }
  const int64_t idx_bytes = (int64_t)sp.idx.size() * 4;
  if (used + idx_bytes <= smem_bytes) {
    sp.idx_in_smem = true;
    used += idx_bytes;
  }
  const int32_t all_units = (int32_t)sp.blobs.size();
  const int64_t extra_desc = 16ll * (all_units - sp.lv_blob_max);
  if (used + extra_desc <= smem_bytes) {
    sp.desc_resident = true;
    sp.lv_blob_max = all_units;
    used += extra_desc;
  }
  sp.smem = (int32_t)used;
  (void)n_cases;
  return JT_OK;
}

int32_t prop_smem_bytes(const Schedule& s, int elem) {
  if (s.cb == kCaseLanes) return SmemLayoutCL(s.ring, s.chunk, s.blob_max, s.win_max).bytes;
  return SmemLayout(s.cb, s.ring, s.chunk, s.max_k, s.max_ports, s.blob_max, s.win_max, elem).bytes;
}

jt_status build_padded_plan(const Plan& p, Plan* q, std::string* err) {
  const int nv = p.n_vars, nc = p.n_cliques;
  std::vector<int32_t> card(nv);
  for (int v = 0; v < nv; ++v) card[v] = (int32_t)(1ll << ilog2(p.card[v]));
  std::vector<int64_t> off(1, 0);
  std::vector<int32_t> vars;
  for (int c = 0; c < nc; ++c) {
    vars.insert(vars.end(), p.vars[c].begin(), p.vars[c].end());
    off.push_back((int64_t)vars.size());
  }
  jt_tree_desc d{};
  d.n_vars = nv;
  d.card = card.data();
  d.n_cliques = nc;
  d.clique_off = off.data();
  d.clique_vars = vars.data();
  d.parent = p.parent.data();
  d.potentials = nullptr;
  d.potentials_dtype = JT_F32;
  d.compute = JT_F32;
  d.max_cases = 1;
  d.flags = 0;
  jt_status st = build_plan(&d, q, err);
  if (st != JT_OK) return st;
  for (int c = 0; c < nc; ++c)
    if (q->pvars[c] != p.pvars[c]) FAIL(JT_ERR_UNSUPPORTED, "padded plan permutes a clique differently");
  // outputs in the original layout: the padded plan writes p's marginal rows
  q->card_ev = p.card;
  q->moff = p.moff;
  q->marg_total = p.marg_total;
  for (int L = 0; L < 3; ++L)
    for (int v = 0; v < nv; ++v) {
      q->vsrc[L][v].moff = p.moff[v];
      q->vsrc[L][v].card_out = p.card[v];
    }
  return JT_OK;
}

PadMap build_pad_map(const Plan& p, const Plan& q) {
  PadMap m;
  for (int c = 0; c < p.n_cliques; ++c) {
    const auto& pv = p.pvars[c];
    const int k = (int)pv.size();
    const int32_t d0 = (int32_t)m.digits.size();
    int64_t st = 1;
    int32_t sh = 0;
    std::vector<int4> dg(k);
    for (int i = k - 1; i >= 0; --i) {
      const int32_t b = ilog2(q.card[pv[i]]);
      dg[i] = int4{sh, b, p.card[pv[i]], (int32_t)st};
      sh += b;
      st *= p.card[pv[i]];
    }
    m.digits.insert(m.digits.end(), dg.begin(), dg.end());
    m.cliques.push_back(PadClique{p.base_off[c], q.base_off[c], q.n_entries[c], d0, k});
  }
  return m;
}

template <typename T>
void permute_tables(const Plan& p, const void* pot, jt_dtype pot_dtype, T* out) {
  // Each clique's table is re-laid out from the listed order to the permuted
  // order: an odometer over the permuted digits tracks the listed index.
  std::vector<int64_t> src_off(p.n_cliques + 1, 0);
  for (int c = 0; c < p.n_cliques; ++c) src_off[c + 1] = src_off[c] + p.n_entries[c];
  auto work = [&](int c) {
    const auto& lv = p.vars[c];
    const auto& pv = p.pvars[c];
    int k = (int)lv.size();
    std::vector<int64_t> lst(k);
    int64_t s = 1;
    for (int i = k - 1; i >= 0; --i) {
      lst[i] = s;
      s *= p.card[lv[i]];
    }
    std::vector<int64_t> pst(k);  // listed stride of each permuted position
    std::vector<int32_t> pc(k);
    for (int i = 0; i < k; ++i) {
      int v = pv[i];
      pc[i] = p.card[v];
      for (int j = 0; j < k; ++j)
        if (lv[j] == v) pst[i] = lst[j];
    }
    std::vector<int32_t> dig(k, 0);
    int64_t src = 0;
    T* dst = out + p.base_off[c];
    const int64_t n = p.n_entries[c];
    const int64_t so = src_off[c];
    for (int64_t e = 0; e < n; ++e) {
      double x = !pot                  ? 1.0
                 : pot_dtype == JT_F64 ? ((const double*)pot)[so + src]
                                       : (double)((const float*)pot)[so + src];
      dst[e] = (T)x;
      for (int i = k - 1; i >= 0; --i) {  // odometer increment
        if (++dig[i] < pc[i]) {
          src += pst[i];
          break;
        }
        dig[i] = 0;
        src -= pst[i] * (pc[i] - 1);
      }
    }
    int64_t padded = (n + 31) / 32 * 32;
    for (int64_t e = n; e < padded; ++e) dst[e] = (T)0;
  };
  int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  std::atomic<int> next{0};
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&] {
      for (int c; (c = next.fetch_add(1)) < p.n_cliques;) work(c);
    });
  for (auto& x : th) x.join();
}

template void permute_tables<float>(const Plan&, const void*, jt_dtype, float*);
template void permute_tables<double>(const Plan&, const void*, jt_dtype, double*);

}  // namespace jt

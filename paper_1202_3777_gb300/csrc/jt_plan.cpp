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

namespace jt {

uint32_t magic_for(uint32_t d) {
  // ceil(2^32 / d); with q = umulhi(n, m) the true quotient is q or q - 1 for
  // every 32-bit n (the kernel corrects with one compare).
  if (d <= 1) return 0;
  return (uint32_t)(((1ull << 32) + d - 1) / d);
}

// Columns kept per row (product of the trailing private cardinalities).
constexpr int64_t kMaxCols = 4096;

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
  if (!d->card || !d->clique_off || !d->clique_vars || !d->parent || !d->potentials)
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
  for (int64_t i = 0; i < p->entries; ++i) {
    double x = d->potentials_dtype == JT_F64 ? ((const double*)d->potentials)[i]
                                             : (double)((const float*)d->potentials)[i];
    if (!(x >= 0.0) || !std::isfinite(x)) FAIL(JT_ERR_INVALID_ARG, "potentials must be finite and >= 0");
  }
  p->work_per_case = 0;
  for (int c = 1; c < nc; ++c) p->work_per_case += 2 * (p->n_entries[c] + p->n_entries[p->parent[c]]);

  // separator tables: root gets a 1-entry slot (its total), edges follow
  p->sep_size.assign(nc, 1);
  p->sep_off.assign(nc, 0);
  int64_t off = 1;
  for (int c = 1; c < nc; ++c) {
    int64_t s = 1;
    for (int v : p->sep[c]) s *= p->card[v];
    p->sep_size[c] = (int32_t)s;
    p->sep_off[c] = (int32_t)off;
    off += s;
    if (off > (1ll << 30)) FAIL(JT_ERR_UNSUPPORTED, "separator tables too large");
  }
  p->msg_total = (int32_t)off;

  // marginal sources: a variable in some separator is read from the smallest
  // such separator after distribution; any other variable lives in exactly
  // one clique and is accumulated there ("home" variables).
  p->moff.assign(nv, 0);
  int64_t mo = 0;
  for (int v = 0; v < nv; ++v) {
    p->moff[v] = (int32_t)mo;
    mo += p->card[v];
  }
  p->marg_total = (int32_t)mo;
  p->home.assign(nv, -1);
  p->src_edge.assign(nv, -1);
  for (int c = 0; c < nc; ++c)
    for (int v : p->vars[c])
      if (holders[v] == 1) p->home[v] = c;
  for (int c = 1; c < nc; ++c)
    for (int v : p->sep[c]) {
      int e = p->src_edge[v];
      if (e < 0 || p->sep_size[c] < p->sep_size[e]) p->src_edge[v] = c;
    }

  // permuted order: parent separator (ascending), variables of child
  // separators (ascending), then the private variables (ascending) -- with a
  // private variable whose cardinality is a multiple of 4 moved last when one
  // exists, so a 4-wide vector of entries stays inside one row.
  p->pvars.assign(nc, {});
  std::vector<int32_t> n_private(nc, 0);
  for (int c = 0; c < nc; ++c) {
    std::vector<int32_t> a = p->sep[c], b, r;
    for (int v : a) mark[v] = 1;
    for (int g : p->children[c])
      for (int v : p->sep[g])
        if (!mark[v]) {
          mark[v] = 2;
          b.push_back(v);
        }
    for (int v : p->vars[c])
      if (!mark[v]) r.push_back(v);
    for (int v : p->vars[c]) mark[v] = 0;
    std::sort(b.begin(), b.end());
    std::sort(r.begin(), r.end());
    std::vector<int32_t>& last = r.empty() ? b : r;
    if (!last.empty() && p->card[last.back()] % 4 != 0) {
      for (size_t i = 0; i < last.size(); ++i)
        if (p->card[last[i]] % 4 == 0) {
          int32_t v = last[i];
          last.erase(last.begin() + i);
          last.push_back(v);
          break;
        }
    }
    n_private[c] = (int32_t)r.size();
    std::vector<int32_t>& pv = p->pvars[c];
    pv.insert(pv.end(), a.begin(), a.end());
    pv.insert(pv.end(), b.begin(), b.end());
    pv.insert(pv.end(), r.begin(), r.end());
  }

  // padded offsets (multiples of 32 elements: 128 B for FP32, 256 B for FP64)
  p->base_off.resize(nc);
  int64_t bo = 0;
  for (int c = 0; c < nc; ++c) {
    p->base_off[c] = bo;
    bo += (p->n_entries[c] + 31) / 32 * 32;
  }
  p->base_len = bo;

  // device descriptors
  p->dcl.resize(nc);
  p->dpos.clear();
  p->dch.clear();
  p->dhm.clear();
  p->dsrc.clear();
  p->djh.clear();
  p->dfld.clear();
  p->fac_collect.assign(nc, 0);
  p->out_dist.assign(nc, 0);
  p->joint_total = 0;
  std::vector<int64_t> st(JT_MAX_CLIQUE_VARS);
  std::vector<int32_t> posof(nv, -1);
  for (int c = 0; c < nc; ++c) {
    const auto& pv = p->pvars[c];
    const int k = (int)pv.size();
    bool pow2 = true;
    for (int v : pv) pow2 = pow2 && is_pow2(p->card[v]);
    // column suffix: trailing private variables while the product stays <= kMaxCols
    int kr = k;
    int64_t P = 1;
    while (kr > k - n_private[c] && P * p->card[pv[kr - 1]] <= kMaxCols) {
      P *= p->card[pv[kr - 1]];
      --kr;
    }
    int64_t s = 1;
    for (int i = k - 1; i >= 0; --i) {
      st[i] = s;
      s *= p->card[pv[i]];
    }
    DevClique& dc = p->dcl[c];
    std::memset(&dc, 0, sizeof(dc));
    dc.base_off = p->base_off[c];
    dc.n = (int32_t)p->n_entries[c];
    dc.k = k;
    dc.kr = kr;
    dc.P = (int32_t)P;
    dc.P_magic = magic_for((uint32_t)P);
    dc.logP = pow2 ? ilog2(P) : 0;
    dc.sep_size = p->sep_size[c];
    dc.sep_off = p->sep_off[c];
    const int64_t L = p->n_entries[c] / p->sep_size[c];
    dc.LR = (int32_t)(L / P);
    dc.LR_magic = magic_for((uint32_t)dc.LR);
    dc.logLR = pow2 ? ilog2(dc.LR) : 0;
    dc.pow2 = pow2 ? 1 : 0;
    dc.depth = p->depth[c];
    dc.card_last = p->card[pv[k - 1]];
    dc.pos_first = (int32_t)p->dpos.size();
    for (int i = 0; i < k; ++i) {
      DevPos q{};
      q.var = pv[i];
      q.card = p->card[pv[i]];
      q.is_col = i >= kr ? 1 : 0;
      const int64_t sti = i >= kr ? st[i] : st[i] / P;   // column stride or row stride
      q.st = (int32_t)sti;
      q.st_magic = magic_for((uint32_t)sti);
      q.card_magic = magic_for((uint32_t)q.card);
      q.sh = pow2 ? ilog2(sti) : 0;
      q.cbits = pow2 ? ilog2(q.card) : 0;
      p->dpos.push_back(q);
      posof[pv[i]] = i;
    }
    // children: digit-run fields of each child separator over the row index
    dc.child_first = (int32_t)p->dch.size();
    dc.n_child = (int32_t)p->children[c].size();
    int32_t fac = 0;
    const int32_t field0 = (int32_t)p->dfld.size();
    for (int g : p->children[c]) {
      const auto& sv = p->sep[g];  // ascending = table order, first most significant
      std::vector<int64_t> ts(sv.size());
      int64_t t = 1;
      for (int i = (int)sv.size() - 1; i >= 0; --i) {
        ts[i] = t;
        t *= p->card[sv[i]];
      }
      std::vector<int64_t> tstride_at(k, 0);
      std::vector<char> in(k, 0);
      for (size_t i = 0; i < sv.size(); ++i) {
        in[posof[sv[i]]] = 1;
        tstride_at[posof[sv[i]]] = ts[i];
      }
      DevChild ch{};
      ch.child = g;
      ch.sep_size = p->sep_size[g];
      ch.sep_off = p->sep_off[g];
      ch.field_first = (int32_t)p->dfld.size();
      ch.field_rel = ch.field_first - field0;
      ch.fac_off = fac;
      ch.w_last = (kr == k && in[k - 1]) ? (int32_t)tstride_at[k - 1] : 0;
      int i = kr - 1;
      while (i >= 0) {
        if (!in[i]) {
          --i;
          continue;
        }
        int j = i;  // run [j, i]
        int64_t len = p->card[pv[i]];
        while (j - 1 >= 0 && in[j - 1] && tstride_at[j - 1] == tstride_at[j] * p->card[pv[j]]) {
          --j;
          len *= p->card[pv[j]];
        }
        DevField f{};
        const int64_t rs = st[i] / P;
        f.st = (int32_t)rs;
        f.len = (int32_t)len;
        f.st_magic = magic_for((uint32_t)rs);
        f.len_magic = magic_for((uint32_t)len);
        f.w = (int32_t)tstride_at[i];
        f.sh = pow2 ? ilog2(rs) : 0;
        f.lbits = pow2 ? ilog2(len) : 0;
        p->dfld.push_back(f);
        i = j - 1;
      }
      ch.n_field = (int32_t)p->dfld.size() - ch.field_first;
      p->dch.push_back(ch);
      fac += ch.sep_size;
    }
    dc.field_first = field0;
    dc.n_field = (int32_t)p->dfld.size() - field0;
    for (int v : pv) posof[v] = -1;
    // private variables at row positions: marginal accumulated per row
    dc.home_first = (int32_t)p->dhm.size();
    int32_t homes = 0;
    for (int i = 0; i < kr; ++i) {
      int v = pv[i];
      if (p->home[v] == c) {
        p->dhm.push_back(DevHome{i, p->card[v], p->moff[v], fac + homes});
        homes += p->card[v];
      }
    }
    dc.n_home = (int32_t)p->dhm.size() - dc.home_first;
    // private variables in the columns: marginal binned from the column joint
    dc.jh_first = (int32_t)p->djh.size();
    for (int i = kr; i < k; ++i) p->djh.push_back(DevSrc{pv[i], p->card[pv[i]], (int32_t)st[i], p->moff[pv[i]]});
    dc.n_jh = (int32_t)p->djh.size() - dc.jh_first;
    dc.joint_off = -1;
    if (P > 1) {
      dc.joint_off = p->joint_total;
      p->joint_total += (int32_t)P;
    }
    // variables read from this clique's parent separator
    dc.src_first = (int32_t)p->dsrc.size();
    if (c > 0) {
      const auto& sv = p->sep[c];
      int64_t t = 1;
      std::vector<int64_t> ts(sv.size());
      for (int i = (int)sv.size() - 1; i >= 0; --i) {
        ts[i] = t;
        t *= p->card[sv[i]];
      }
      for (size_t i = 0; i < sv.size(); ++i)
        if (p->src_edge[sv[i]] == c) p->dsrc.push_back(DevSrc{sv[i], p->card[sv[i]], (int32_t)ts[i], p->moff[sv[i]]});
    }
    dc.n_src = (int32_t)p->dsrc.size() - dc.src_first;
    p->fac_collect[c] = fac;
    p->out_dist[c] = fac + homes;
  }
  // marginal sources, as offsets in the per-case array
  // [up | down | rho | marg | joint] (see LevelArgs)
  p->vsrc.assign(nv, VarSrc{});
  for (int v = 0; v < nv; ++v) {
    VarSrc& q = p->vsrc[v];
    q.card = p->card[v];
    q.moff = p->moff[v];
    const int e = p->src_edge[v];
    if (e >= 0) {           // separator-held: bin the distribute message of edge e
      q.kind = 1;
      q.off = (int64_t)p->msg_total + p->sep_off[e];
      q.size = p->sep_size[e];
      int64_t t = 1;
      for (int i = (int)p->sep[e].size() - 1; i >= 0; --i) {
        if (p->sep[e][i] == v) q.st = (int32_t)t;
        t *= p->card[p->sep[e][i]];
      }
      continue;
    }
    const int c = p->home[v];
    const DevClique& dc = p->dcl[c];
    int pos = -1;
    for (int i = 0; i < dc.k; ++i)
      if (p->pvars[c][i] == v) pos = i;
    if (pos >= dc.kr) {     // in the column joint of its clique
      q.kind = 1;
      q.off = 3ll * p->msg_total + p->marg_total + dc.joint_off;
      q.size = dc.P;
      q.st = p->dpos[dc.pos_first + pos].st;
    } else {                // accumulated per row
      q.kind = 0;
      q.off = 3ll * p->msg_total + p->moff[v];
    }
  }
  return JT_OK;
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
      double x = pot_dtype == JT_F64 ? ((const double*)pot)[so + src] : (double)((const float*)pot)[so + src];
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

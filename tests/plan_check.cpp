#include <array>
// Host-side check of the propagation planner (no GPU): builds the plan and
// the schedules of a tree read from stdin and checks the invariants the
// persistent kernel relies on.
//
//   * Every block of every stage is one work item per case block, and the
//     items tile the stage's table.
//   * Dependencies follow Algorithms 2-4: a collect stage waits for every
//     child's collect stage, the root's distribute stage for every child's
//     collect stage, any other distribute stage for its parent's distribute
//     stage, each for all of that stage's blocks.
//   * Work items are claimed in queue order and an item waits only for the
//     blocks it depends on, so the kernel cannot wait forever on work no
//     CTA has claimed: every block an item waits for comes earlier in the
//     queue.
//
// Input (whitespace-separated integers): n_vars, card[n_vars], n_cliques,
// then per clique k followed by its k variables, then parent[n_cliques].
// With "plant-inchunk" every one-case port is claimed to keep its key over a
// chunk's iterations (the check must then fail on trees whose blocks span
// several iterations).
// With argument "plant-order" the queue is reversed, with "plant-repeat" one
// item is queued twice, before the checks (each must then fail).
// Output: one line per (case-block width, case count):
//   "cb=<cb> cases=<n> OK items=<i> stages=<s>" or "... UNSUPPORTED <why>" or
//   "... FAIL <what>".
#include <algorithm>
#include <cstdio>
#include <iostream>
#include <string>
#include <vector>

#include "jt_internal.h"
#include "jt_kernels.h"

using namespace jt;

namespace {

std::string check(const Plan& p, const Schedule& s) {
  const int nc = p.n_cliques;
  const int nst = (int)s.stages.size();
  if (nst != 2 * nc) return "stage count";
  // tiling: per (stage, case block) every block exactly once
  std::vector<std::vector<int>> seen((size_t)nst * s.n_cb);
  for (const DevItem& it : s.items) {
    if (it.stage < 0 || it.stage >= nst || it.cbk < 0 || it.cbk >= s.n_cb) return "item index out of range";
    const DevStage& S = s.stages[it.stage];
    if (it.block < 0 || it.block >= S.n_blocks) return "block out of range";
    if (it.off != S.base_off + (int64_t)it.block * S.B || it.n != S.B) return "item does not tile its stage";
    seen[(size_t)it.stage * s.n_cb + it.cbk].push_back(it.block);
  }
  for (int st = 0; st < nst; ++st) {
    const DevStage& S = s.stages[st];
    if (S.n_blocks > 0 && ((int64_t)S.n_blocks * S.B < S.n || (int64_t)(S.n_blocks - 1) * S.B >= S.n))
      return "blocks do not cover stage " + std::to_string(st);
    for (int q = 0; q < s.n_cb; ++q) {
      std::vector<int> b = seen[(size_t)st * s.n_cb + q];
      if ((int)b.size() != S.n_blocks) return "stage " + std::to_string(st) + " has a missing or repeated block";
      std::vector<char> got(S.n_blocks, 0);
      for (int x : b) {
        if (got[x]) return "repeated block";
        got[x] = 1;
      }
    }
  }
  // dependencies as Algorithms 2-4 order them
  for (int pass = 0; pass < 2; ++pass)
    for (int c = 0; c < nc; ++c) {
      const DevStage& S = s.stages[pass * nc + c];
      std::vector<std::pair<int, int>> want;
      if (pass == 0 || c == 0) {
        if (!(pass == 0 && c == 0))
          for (int g : p.children[c]) want.push_back({g, s.stages[g].n_blocks});
      } else {
        want.push_back({nc + p.parent[c], s.stages[nc + p.parent[c]].n_blocks});
      }
      if (S.ndep != (int)want.size()) return "dependency count of stage " + std::to_string(pass * nc + c);
      for (int i = 0; i < S.ndep; ++i)
        if (s.deps[S.dep0 + 2 * i] != want[i].first || s.deps[S.dep0 + 2 * i + 1] != want[i].second)
          return "dependency of stage " + std::to_string(pass * nc + c);
    }
  // case-lane schedules: every block holds whole tiles of 32 entries and at
  // most kClMaxChunks chunks, on the power-of-two path
  if (s.cb == kCaseLanes)
    for (const DevStage& S : s.stages) {
      if (S.n_blocks == 0) continue;
      if (S.bits < 5 || S.B != (1 << S.bits)) return "case-lane block of stage " + std::to_string(&S - &s.stages[0]);
      if ((S.B + s.chunk - 1) / s.chunk > kClMaxChunks) return "case-lane block longer than the chunk table";
    }
  // queue order: the blocks an item waits for are all claimed before it
  std::vector<int> done((size_t)nst * s.n_cb, 0);
  for (size_t i = 0; i < s.items.size(); ++i) {
    const DevItem& it = s.items[i];
    const DevStage& S = s.stages[it.stage];
    for (int d = 0; d < S.ndep; ++d) {
      const int st = s.deps[S.dep0 + 2 * d], need = s.deps[S.dep0 + 2 * d + 1];
      if (done[(size_t)st * s.n_cb + it.cbk] < need)
        return "item " + std::to_string(i) + " waits for blocks queued after it";
    }
    ++done[(size_t)it.stage * s.n_cb + it.cbk];
  }
  // one case: a port not marked as depending on the iteration bits inside a
  // chunk has one key for all of a thread's vectors of the chunk (the kernel
  // gathers and reduces them once), and one not marked as depending on the
  // iteration has one key for the whole block (FP32 plans: four entries per
  // vector)
  if (s.cb == 1) {
    const int ipc = std::max<int>(1, (int)(s.chunk / (consumers_for(1) * 4)));
    std::vector<char> seen_st(s.stages.size(), 0);
    for (const DevItem& it : s.items) {
      if (seen_st[it.stage]) continue;
      seen_st[it.stage] = 1;
      const DevStage& S = s.stages[it.stage];
      if (S.bits < 0 || S.n_live == 0) continue;
      const unsigned char* blob = reinterpret_cast<const unsigned char*>(s.blobs.data()) + (size_t)it.blob * 16;
      const LivePort* lp = reinterpret_cast<const LivePort*>(blob + S.live_off);
      const int32_t* ki = reinterpret_cast<const int32_t*>(blob + kiter_off(S));
      for (int li = 0; li < S.n_live; ++li) {
        const int32_t* k = ki + (size_t)li * kMaxIter;
        for (int m = 0; m < S.n_iter; ++m) {
          if (!(lp[li].mode & kModeInChunk) && k[m] != k[m / ipc * ipc])
            return "stage of clique " + std::to_string(S.clique) + " shares a key that varies inside a chunk";
          if (!(lp[li].mode & kModeIter) && k[m] != k[0])
            return "stage of clique " + std::to_string(S.clique) + " has an iteration-free key that varies";
        }
      }
    }
  }
  // case lanes: an output marked for register accumulation must have the
  // same four rows in every tile of its block (a key over entry bits 0-1
  // only), and be no input
  if (s.cb == kCaseLanes)
    for (const DevItem& it : s.items) {
      const DevStage& S = s.stages[it.stage];
      const unsigned char* blob = reinterpret_cast<const unsigned char*>(s.blobs.data()) + (size_t)it.blob * 16;
      const CLPort* cp = reinterpret_cast<const CLPort*>(blob + S.live_off);
      int marked = 0;
      for (int li = 0; li < S.n_live; ++li) {
        const CLPort& C = cp[li];
        if (((C.cls >> kClRegShift) & 3) == 0) continue;
        ++marked;
        bool same = (C.cls & kClInput) == 0 && (C.dep & ~3) == 0 && (C.cls & kClEntry) != 0;
        for (int q = 1; q < 64; ++q) same = same && C.kslot[q] == C.kslot[0];
        for (int q = 1; q < kClMaxChunks; ++q) same = same && C.kchunk[q] == C.kchunk[0];
        if (!same) return "stage of clique " + std::to_string(S.clique) + " accumulates an output whose rows vary";
      }
      if (marked > kClRegSlots) return "more register-accumulated outputs than slots";
    }
  return "";
}

}  // namespace

int main(int argc, char** argv) {
  const std::string plant = argc > 1 ? argv[1] : "";
  int nv = 0, nc = 0;
  if (!(std::cin >> nv) || nv <= 0) return 2;
  std::vector<int32_t> card(nv);
  for (auto& x : card) std::cin >> x;
  std::cin >> nc;
  std::vector<int64_t> off(1, 0);
  std::vector<int32_t> vars;
  for (int c = 0; c < nc; ++c) {
    int k = 0;
    std::cin >> k;
    for (int i = 0; i < k; ++i) {
      int v = 0;
      std::cin >> v;
      vars.push_back(v);
    }
    off.push_back((int64_t)vars.size());
  }
  std::vector<int32_t> parent(nc);
  for (auto& x : parent) std::cin >> x;
  if (!std::cin) return 2;
  jt_tree_desc d{};
  d.n_vars = nv;
  d.card = card.data();
  d.n_cliques = nc;
  d.clique_off = off.data();
  d.clique_vars = vars.data();
  d.parent = parent.data();
  d.potentials = nullptr;
  d.potentials_dtype = JT_F64;
  d.compute = JT_F32;
  d.max_cases = 64;
  Plan p;
  std::string err;
  if (build_plan(&d, &p, &err) != JT_OK) {
    std::printf("PLAN FAIL %s\n", err.c_str());
    return 1;
  }
  const int smem = 232448 - 256;  // the opt-in shared memory of one CTA on this GPU, less the reserve
  const int shapes[][2] = {{1, 1}, {4, 16}, {8, 16}, {8, 64}, {kCaseLanes, 64}, {kCaseLanes, 40}};
  int bad = 0;
  for (const auto& sh : shapes) {
    Schedule s;
    err.clear();
    const jt_status st = build_schedule(p, 4, sh[0], sh[1], 152, smem, &s, &err);
    if (st == JT_ERR_UNSUPPORTED) {
      std::printf("cb=%d cases=%d UNSUPPORTED %s\n", sh[0], sh[1], err.c_str());
      continue;
    }
    if (st != JT_OK) {
      std::printf("cb=%d cases=%d FAIL status %d %s\n", sh[0], sh[1], (int)st, err.c_str());
      ++bad;
      continue;
    }
    if (plant == "plant-order") std::reverse(s.items.begin(), s.items.end());
    if (plant == "plant-repeat" && s.items.size() > 1) s.items.back() = s.items.front();
    if (plant == "plant-inchunk" && s.cb == 1)  // every port claimed to share its key inside a chunk
      for (const DevItem& it : s.items) {
        const DevStage& S = s.stages[it.stage];
        if (S.bits < 0) continue;
        LivePort* lp = reinterpret_cast<LivePort*>(reinterpret_cast<unsigned char*>(s.blobs.data()) +
                                                   (size_t)it.blob * 16 + S.live_off);
        for (int li = 0; li < S.n_live; ++li) lp[li].mode &= ~kModeInChunk;
      }
    const std::string why = check(p, s);
    if (why.empty()) {
      std::printf("cb=%d cases=%d OK items=%zu stages=%zu\n", sh[0], sh[1], s.items.size(), s.stages.size());
    } else {
      std::printf("cb=%d cases=%d FAIL %s\n", sh[0], sh[1], why.c_str());
      ++bad;
    }
  }
  // block targets scaled per clique-size class (the autotuner's search
  // space): the same invariants hold, and a shift moves the block sizes
  for (int d : {-1, 1}) {
    const int8_t sh[kBlockClasses] = {(int8_t)d, (int8_t)d, (int8_t)d};
    for (const auto& shp : {std::array<int, 2>{1, 1}, std::array<int, 2>{8, 64}}) {
      Schedule s;
      err.clear();
      const jt_status st = build_schedule(p, 4, shp[0], shp[1], 152, smem, &s, &err, sh);
      if (st == JT_ERR_UNSUPPORTED) continue;
      std::string why = st == JT_OK ? check(p, s) : "status " + std::to_string((int)st) + " " + err;
      for (int q = 0; q < kBlockClasses && why.empty(); ++q)
        if (s.block_shift[q] != d) why = "shift not recorded";
      if (why.empty()) {
        std::printf("tune shift=%d cb=%d cases=%d OK items=%zu\n", d, shp[0], shp[1], s.items.size());
      } else {
        std::printf("tune shift=%d cb=%d cases=%d FAIL %s\n", d, shp[0], shp[1], why.c_str());
        ++bad;
      }
    }
  }
  // the whole-tree plan: the packed indices unpack to the plan's arrays, and
  // a collect stage's scale (written in the first phase of the level after
  // its own) is ready before its parent's collect level runs
  {
    Schedule s;
    err.clear();
    const jt_status st = build_small_schedule(p, 4, 64, 152, smem, &s, &err);
    if (st == JT_ERR_UNSUPPORTED) {
      std::printf("small UNSUPPORTED %s\n", err.c_str());
    } else if (st != JT_OK) {
      std::printf("small FAIL status %d %s\n", (int)st, err.c_str());
      ++bad;
    } else {
      const auto& sp = s.small;
      std::string why;
      auto same = [&](int32_t o, const std::vector<int32_t>& v, const char* what) {
        for (size_t i = 0; i < v.size() && why.empty(); ++i)
          if (sp.idx[o + i] != v[i]) why = std::string("packed ") + what + " differs";
      };
      same(0, sp.lv_blob_off, "lv_blob_off");
      same(sp.o_seg_lv, sp.seg_lv, "seg_lv");
      same(sp.o_lv_stage_off, sp.lv_stage_off, "lv_stage_off");
      same(sp.o_stage_blob, sp.stage_blob, "stage_blob");
      same(sp.o_lv_stage, sp.lv_stage, "lv_stage");
      same(sp.o_sep_size, p.sep_size, "sep_size");
      for (size_t i = 0; i < sp.segs.size() && why.empty(); ++i)
        if (sp.idx[sp.o_segs + 2 * i] != sp.segs[i].x || sp.idx[sp.o_segs + 2 * i + 1] != sp.segs[i].y)
          why = "packed segs differ";
      if (why.empty() && (sp.idx.size() % 4 || sp.o_segs % 2)) why = "packed layout misaligned";
      std::vector<int> level_of(2 * nc, -1);
      for (int lv = 0; lv < sp.levels; ++lv)
        for (int j = sp.lv_stage_off[lv]; j < sp.lv_stage_off[lv + 1]; ++j) level_of[sp.lv_stage[j]] = lv;
      for (int c = 1; c < nc && why.empty(); ++c) {
        const int par = p.parent[c];
        const int lc = level_of[c], lp = par == 0 ? level_of[nc] : level_of[par];
        if (lc < 0 || lp < 0 || lp <= lc)
          why = "collect of clique " + std::to_string(c) + " is not before its parent's stage";
      }
      if (why.empty() && sp.smem > smem) why = "shared memory over budget";
      if (why.empty()) {
        std::printf("small OK levels=%d segs=%zu smem=%d idx_in_smem=%d desc_resident=%d\n", sp.levels,
                    sp.segs.size(), sp.smem, (int)sp.idx_in_smem, (int)sp.desc_resident);
      } else {
        std::printf("small FAIL %s\n", why.c_str());
        ++bad;
      }
    }
  }
  // trees with other cardinalities: the power-of-two padded plan, its
  // case-lane schedules, and the map that derives its tables
  if (std::any_of(p.pow2.begin(), p.pow2.end(), [](uint8_t x) { return x == 0; })) {
    Plan q;
    err.clear();
    if (build_padded_plan(p, &q, &err) != JT_OK) {
      std::printf("pad FAIL plan %s\n", err.c_str());
      return 1;
    }
    for (int cases : {64, 40}) {
      Schedule s;
      err.clear();
      const jt_status st = build_schedule(q, 4, kCaseLanes, cases, 152, smem, &s, &err);
      if (st == JT_ERR_UNSUPPORTED) {
        std::printf("pad cb=%d cases=%d UNSUPPORTED %s\n", kCaseLanes, cases, err.c_str());
        continue;
      }
      if (plant == "plant-order") std::reverse(s.items.begin(), s.items.end());
      if (plant == "plant-repeat" && s.items.size() > 1) s.items.back() = s.items.front();
      if (plant == "plant-holes")   // one state too few: the last real state reads as added
        for (DevStage& S : s.stages)
          if (S.holes[0] != 0u) S.holes[0] -= 1u << 10;
      std::string why = st == JT_OK ? check(q, s) : "status " + std::to_string((int)st) + " " + err;
      // evidence limits and output rows are the original tree's
      for (const DevPos& P : s.pos)
        if (why.empty() && P.card_ev != p.card[P.var]) why = "evidence limit of a padded digit";
      // a tile the stage marks as holes (a digit above it at an added state)
      // must hold only entries with some digit at an added state
      int64_t tiles = 0, skipped = 0;
      for (const DevStage& S : s.stages) {
        if (S.n_blocks == 0 || !why.empty()) continue;
        const auto& pv = q.pvars[S.clique];
        for (int64_t x0 = 0; x0 < S.n && why.empty(); x0 += 32) {
          ++tiles;
          bool flagged = false;
          for (uint32_t h : S.holes)
            if (h != 0u && ((x0 >> (h & 31u)) & ((1ll << ((h >> 5) & 31u)) - 1)) >= (int64_t)(h >> 10)) flagged = true;
          if (!flagged) continue;
          ++skipped;
          for (int64_t e = x0; e < x0 + 32 && why.empty(); ++e) {
            int64_t r = e;
            bool hole = false;
            for (int i = (int)pv.size() - 1; i >= 0; --i) {
              if (r % q.card[pv[i]] >= p.card[pv[i]]) hole = true;
              r /= q.card[pv[i]];
            }
            if (!hole) why = "tile at " + std::to_string(x0) + " of clique " + std::to_string(S.clique) +
                             " marked as holes holds entry " + std::to_string(e);
          }
        }
      }
      if (why.empty()) {
        std::printf("pad cb=%d cases=%d OK items=%zu hole-tiles=%.3f\n", kCaseLanes, cases, s.items.size(),
                    tiles ? (double)skipped / tiles : 0.0);
      } else {
        std::printf("pad cb=%d cases=%d FAIL %s\n", kCaseLanes, cases, why.c_str());
        ++bad;
      }
    }
    std::string why;
    if (q.moff != p.moff || q.marg_total != p.marg_total) why = "marginal rows differ";
    for (int v = 0; v < nv && why.empty(); ++v)
      if (q.vsrc[2][v].card_out != p.card[v] || q.card[v] < p.card[v] || (q.card[v] & (q.card[v] - 1)))
        why = "padded cardinality or output states of variable " + std::to_string(v);
    // every padded entry, decoded by its own digits: the map must find the
    // original entry with the same digits, or a hole where a digit is padded
    PadMap m = build_pad_map(p, q);
    if (plant == "plant-pad" && m.digits.size() > 1) std::swap(m.digits[0].w, m.digits[1].w);
    int64_t holes = 0, kept = 0;
    for (int c = 0; c < nc && why.empty(); ++c) {
      const auto& pv = q.pvars[c];
      const int k = (int)pv.size();
      const PadClique& pc = m.cliques[c];
      if (pc.k != k || pc.off != p.base_off[c] || pc.off_pad != q.base_off[c] || pc.n_pad != q.n_entries[c]) {
        why = "clique record of clique " + std::to_string(c);
        break;
      }
      for (int64_t e = 0; e < q.n_entries[c] && why.empty(); ++e) {
        int64_t r = e, want = 0, st = 1;
        bool hole = false;
        for (int i = k - 1; i >= 0; --i) {
          const int64_t dgt = r % q.card[pv[i]];
          r /= q.card[pv[i]];
          if (dgt >= p.card[pv[i]]) hole = true;
          want += dgt * st;
          st *= p.card[pv[i]];
        }
        int64_t got = 0;
        bool ghole = false;
        for (int i = 0; i < k; ++i) {
          const int4 g = m.digits[pc.d0 + i];
          const int64_t dgt = (e >> g.x) & ((1ll << g.y) - 1);
          ghole |= dgt >= g.z;
          got += dgt * g.w;
        }
        if (hole != ghole || (!hole && got != want))
          why = "padded entry " + std::to_string(e) + " of clique " + std::to_string(c);
        hole ? ++holes : ++kept;
      }
    }
    if (why.empty() && kept != p.entries) why = "kept entries " + std::to_string(kept);
    if (why.empty()) {
      std::printf("padmap OK kept=%lld holes=%lld\n", (long long)kept, (long long)holes);
    } else {
      std::printf("padmap FAIL %s\n", why.c_str());
      ++bad;
    }
  }
  return bad ? 1 : 0;
}

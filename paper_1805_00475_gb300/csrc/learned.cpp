// Learned contraction ordering: a greedy merge loop whose choice among the
// candidate merges is made by a small learned edge scorer (mlp.cu), trained
// on plan costs the method itself measures, with the paper's heuristics
// (Sec. 3.1.1) as fallback and as the judge of the cost.
//
// State: the live tensors of a partial contraction and, for every pair of
// live tensors joined by bonds, the number of bonds they share.  A candidate
// is such a pair; merging it follows the edge-contraction rule of Sec. 2.2.
// Label of a candidate (training): its regret, i.e. log2 of the total MACs of
// the plan obtained by merging it and finishing with tensor-greedy, minus the
// smallest such value among the state's candidates.  The scorer predicts the
// regret; the learned plan merges the candidate with the smallest prediction.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "tnc_internal.h"

namespace tnc {

int mlp_forward_bf16_dev(const void* Pb, const float* X, int64_t rows, float* Y, void* stream);
int finish_plan(tnc_plan_t* p, int rank_cap, tnc_plan_stats* stats);
void copy_device(void* dst, const void* src, size_t bytes, int dir, void* stream, int* rc);

namespace {

struct Cand {
  int a, b, k;
};

struct GState {
  Tree t;
  std::vector<char> live;
  std::vector<std::map<int, int>> nb;  // live node -> (live neighbour -> shared bonds)
  int n_live = 0, n_leaves = 0, max_rank = 0;
  double macs = 0.0;

  void init(const Network& net) {
    t = Tree();
    t.n_leaves = net.n_leaves();
    t.nodes.resize(net.n_leaves());
    for (int i = 0; i < net.n_leaves(); i++) {
      t.nodes[i].bonds = net.leaves[i].bonds;
      std::sort(t.nodes[i].bonds.begin(), t.nodes[i].bonds.end());
      max_rank = std::max(max_rank, (int)t.nodes[i].bonds.size());
    }
    t.root = net.n_leaves() == 1 ? 0 : -1;
    n_leaves = net.n_leaves();
    live.assign(2 * n_leaves + 2, 0);
    nb.assign(2 * n_leaves + 2, {});
    for (int i = 0; i < n_leaves; i++) live[i] = 1;
    n_live = n_leaves;
    for (int b = 0; b < net.n_bonds; b++) {
      const int u = net.bond_end0[b], v = net.bond_end1[b];
      if (u < 0 || v < 0 || u == v) continue;
      nb[u][v]++;
      nb[v][u]++;
    }
    macs = 0.0;
  }
  int rank(int i) const { return (int)t.nodes[i].bonds.size(); }
  void merge(int a, int b) {
    if (a > b) std::swap(a, b);
    Node n;
    n.left = a;
    n.right = b;
    std::set_symmetric_difference(t.nodes[a].bonds.begin(), t.nodes[a].bonds.end(), t.nodes[b].bonds.begin(),
                                  t.nodes[b].bonds.end(), std::back_inserter(n.bonds));
    const int k = (rank(a) + rank(b) - (int)n.bonds.size()) / 2;
    macs += std::ldexp(1.0, rank(a) + rank(b) - k);
    t.nodes.push_back(std::move(n));
    const int c = (int)t.nodes.size() - 1;
    t.root = c;
    max_rank = std::max(max_rank, rank(c));
    live[a] = live[b] = 0;
    live[c] = 1;
    n_live--;
    std::map<int, int> nc;
    for (int src : {a, b})
      for (auto& kv : nb[src])
        if (kv.first != a && kv.first != b) nc[kv.first] += kv.second;
    for (auto& kv : nc) {
      auto& m = nb[kv.first];
      m.erase(a);
      m.erase(b);
      m[c] = kv.second;
    }
    nb[c] = std::move(nc);
    nb[a].clear();
    nb[b].clear();
  }
  void candidates(std::vector<Cand>& out) const {
    out.clear();
    for (size_t i = 0; i < t.nodes.size(); i++) {
      if (!live[i]) continue;
      for (auto& kv : nb[i])
        if (kv.first > (int)i) out.push_back({(int)i, kv.first, kv.second});
    }
  }
  // tensor-greedy to the end: smallest result rank, then fewest MACs, then ids;
  // disconnected leftovers joined smallest rank first
  void finish_greedy() {
    std::vector<Cand> cs;
    for (;;) {
      candidates(cs);
      if (cs.empty()) break;
      const Cand* best = nullptr;
      long br = 0, bm = 0;
      for (const Cand& c : cs) {
        const long r = rank(c.a) + rank(c.b) - 2 * c.k, m = rank(c.a) + rank(c.b) - c.k;
        if (!best || r < br || (r == br && (m < bm || (m == bm && (c.a < best->a || (c.a == best->a && c.b < best->b)))))) {
          best = &c;
          br = r;
          bm = m;
        }
      }
      merge(best->a, best->b);
    }
    std::vector<int> rest;
    for (size_t i = 0; i < t.nodes.size(); i++)
      if (live[i]) rest.push_back((int)i);
    while (rest.size() > 1) {
      std::sort(rest.begin(), rest.end(), [&](int x, int y) {
        return rank(x) != rank(y) ? rank(x) < rank(y) : x < y;
      });
      merge(rest[0], rest[1]);
      rest.erase(rest.begin(), rest.begin() + 2);
      rest.push_back((int)t.nodes.size() - 1);
    }
    if (rest.size() == 1) t.root = rest[0];
  }
  double cost() const { return macs > 0 ? std::log2(macs) : 0.0; }
};

// The candidates the scorer sees: the `cap` with the smallest result rank
// (then fewest MACs, then ids).
void top_candidates(const GState& s, std::vector<Cand>& cs, int cap) {
  s.candidates(cs);
  auto key = [&](const Cand& c) {
    return std::make_tuple(s.rank(c.a) + s.rank(c.b) - 2 * c.k, s.rank(c.a) + s.rank(c.b) - c.k, c.a, c.b);
  };
  std::sort(cs.begin(), cs.end(), [&](const Cand& x, const Cand& y) { return key(x) < key(y); });
  if ((int)cs.size() > cap) cs.resize(cap);
}

// The network of the live tensors of a partial contraction: one leaf per
// live tensor (its bonds), every bond between the two live tensors holding it
// (bonds already contracted belong to no live tensor).  Only the structure
// the planners read is set.  ids[j] = tree node of coarse leaf j.
void coarse_network(const GState& s, const Network& net, Network& out, std::vector<int>& ids) {
  out = Network();
  ids.clear();
  for (size_t i = 0; i < s.t.nodes.size(); i++)
    if (s.live[i]) ids.push_back((int)i);
  out.leaves.resize(ids.size());
  out.n_bonds = net.n_bonds;
  out.bond_end0.assign(net.n_bonds, -1);
  out.bond_end1.assign(net.n_bonds, -1);
  out.n_vars = 0;
  out.n_cons = (int)ids.size();
  for (size_t j = 0; j < ids.size(); j++) {
    out.leaves[j].bonds = s.t.nodes[ids[j]].bonds;
    for (int b : out.leaves[j].bonds) {
      if (out.bond_end0[b] < 0) out.bond_end0[b] = (int)j;
      else out.bond_end1[b] = (int)j;
    }
  }
}

// Finishes a partial contraction by the heuristic `h` planned on the network
// of its live tensors (the paper's planners on the coarsened network); h =
// TNC_PLAN_GREEDY is tensor-greedy's own finish.
void complete_with(GState& s, const Network& net, const tnc_plan_opts& h) {
  if (h.heuristic == TNC_PLAN_GREEDY) {
    s.finish_greedy();
    return;
  }
  Network cn;
  std::vector<int> ids;
  coarse_network(s, net, cn, ids);
  if (ids.size() <= 1) {
    s.finish_greedy();
    return;
  }
  Tree ct;
  if (plan_tree(cn, h, ct) != TNC_OK) {
    s.finish_greedy();
    return;
  }
  std::vector<int> map(ct.nodes.size(), -1);
  for (int j = 0; j < ct.n_leaves; j++) map[j] = ids[j];
  for (size_t i = ct.n_leaves; i < ct.nodes.size(); i++) {
    s.merge(map[ct.nodes[i].left], map[ct.nodes[i].right]);
    map[i] = (int)s.t.nodes.size() - 1;
  }
  s.t.root = map[ct.root >= 0 ? ct.root : 0];
}

bool cheaper_cost(const TreeCost& a, const TreeCost& b) {
  return a.max_rank != b.max_rank ? a.max_rank < b.max_rank : a.macs < b.macs;
}

int live_max_rank(const GState& s) {
  int m = 0;
  for (size_t i = 0; i < s.t.nodes.size(); i++)
    if (s.live[i]) m = std::max(m, s.rank((int)i));
  return m;
}

// 16 features of candidate c in state s (scaled to O(1)); live_max is the
// largest rank among the state's live tensors, pos the candidate's position in
// the tensor-greedy order of the state's candidates (0 = greedy's choice).
void features(const GState& s, const Cand& c, int live_max, int pos, int n_cands, float* f) {
  const int ra = s.rank(c.a), rb = s.rank(c.b), k = c.k;
  const int r = ra + rb - 2 * k, lm = ra + rb - k;
  const int da = (int)s.nb[c.a].size(), db = (int)s.nb[c.b].size();
  int touch = 0;
  for (auto& kv : s.nb[c.a])
    if (kv.first != c.b) touch++;
  for (auto& kv : s.nb[c.b])
    if (kv.first != c.a && !s.nb[c.a].count(kv.first)) touch++;
  f[0] = ra / 32.f;
  f[1] = rb / 32.f;
  f[2] = k / 16.f;
  f[3] = r / 32.f;
  f[4] = lm / 64.f;
  f[5] = (r - std::max(ra, rb)) / 16.f;
  f[6] = da / 16.f;
  f[7] = db / 16.f;
  f[8] = pos == 0 ? 1.f : 0.f;
  f[9] = (r - s.max_rank) / 16.f;
  f[10] = 1.f - (float)s.n_live / (float)std::max(1, s.n_leaves);
  f[11] = c.a < s.n_leaves ? 1.f : 0.f;
  f[12] = c.b < s.n_leaves ? 1.f : 0.f;
  f[13] = touch / 16.f;
  f[14] = (r - live_max) / 16.f;
  f[15] = (float)pos / (float)std::max(1, n_cands);
}

struct Rng {
  uint64_t s;
  explicit Rng(uint64_t seed) : s(seed) {}
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
};

}  // namespace

// Training rows: at `states` points of an exploring greedy trajectory of each
// formula, every candidate (at most `cands`) gets its features and its regret.
// With `policy` set, the trajectory follows instead the choices recorded in
// policy[i] (merge sequences of a previous learned plan, as candidate
// positions), so that the scorer also learns on the states it visits itself.
int learned_dataset(const std::vector<const Network*>& nets, int states, int cands, uint64_t seed, std::vector<float>& X,
                    std::vector<float>& T, const std::vector<std::vector<int>>* policy = nullptr,
                    const tnc_plan_opts* completion = nullptr, int max_pct = 100) {
  const int n = (int)nets.size();
  std::vector<std::vector<float>> xs(n), ts(n);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < n; i++) {
    Rng rng(seed ^ (0x5851F42D4C957F2Dull * (uint64_t)(i + 1)));
    GState s;
    s.init(*nets[i]);
    const int steps = std::max(1, (nets[i]->n_leaves() - 1) * std::min(std::max(max_pct, 1), 100) / 100);
    std::vector<int> at;
    for (int j = 0; j < states; j++) at.push_back((int)(rng.next() % (uint64_t)steps));
    std::sort(at.begin(), at.end());
    std::vector<Cand> cs;
    size_t next = 0;
    for (int step = 0;; step++) {
      top_candidates(s, cs, cands);
      if (cs.empty()) break;
      if (next < at.size() && at[next] <= step && cs.size() > 1) {
        while (next < at.size() && at[next] <= step) next++;
        std::vector<double> cost(cs.size());
        for (size_t c = 0; c < cs.size(); c++) {
          GState r = s;
          r.merge(cs[c].a, cs[c].b);
          if (completion) complete_with(r, *nets[i], *completion);
          else r.finish_greedy();
          cost[c] = r.cost();
        }
        const double lo = *std::min_element(cost.begin(), cost.end());
        const int lm = live_max_rank(s);
        for (size_t c = 0; c < cs.size(); c++) {
          float f[TNC_MLP_FEATURES];
          features(s, cs[c], lm, (int)c, (int)cs.size(), f);
          xs[i].insert(xs[i].end(), f, f + TNC_MLP_FEATURES);
          ts[i].push_back((float)(cost[c] - lo));
        }
      }
      // explore: mostly the greedy choice (or the recorded policy's), sometimes one of the next three
      size_t pick = 0;
      if (policy && step < (int)(*policy)[i].size()) pick = std::min<size_t>((size_t)(*policy)[i][step], cs.size() - 1);
      if (cs.size() > 1 && rng.next() % 4 == 0) pick = 1 + rng.next() % std::min<size_t>(3, cs.size() - 1);
      s.merge(cs[pick].a, cs[pick].b);
      if (next >= at.size() && completion) break;  // the states past the last sampled one are not needed
    }
  }
  X.clear();
  T.clear();
  for (int i = 0; i < n; i++) {
    X.insert(X.end(), xs[i].begin(), xs[i].end());
    T.insert(T.end(), ts[i].begin(), ts[i].end());
  }
  return TNC_OK;
}

// Learned plans for many formulas in lockstep: every round gathers the
// candidates of all unfinished formulas, scores them in one bf16 inference
// launch, and merges each formula's lowest predicted regret.
//
// With `completion` set, the learned merges only coarsen the network: at each
// checkpoint (pcts[j] % of the formula's merges) the partial contraction is
// finished by the heuristic `completion` planned on the network of its live
// tensors, and the cheapest (max rank, MACs) of these plans is kept.  Without
// d_params_bf16 the merges follow tensor-greedy's choice (the same loop with
// no scorer: the ablation of the learned part).
int learned_trees(const std::vector<const Network*>& nets, const void* d_params_bf16, void* d_ws, size_t ws_bytes,
                  void* stream, int cands, std::vector<Tree>& trees, std::vector<std::vector<int>>* chosen = nullptr,
                  const tnc_plan_opts* completion = nullptr, const std::vector<int>* pcts = nullptr) {
  const int n = (int)nets.size();
  std::vector<GState> st(n);
  for (int i = 0; i < n; i++) st[i].init(*nets[i]);
  // checkpoints (merge counts) per formula, and the snapshots taken there
  std::vector<std::vector<int>> marks(n);
  std::vector<std::vector<GState>> snaps(n);
  std::vector<int> merged(n, 0);
  if (completion && pcts)
    for (int i = 0; i < n; i++) {
      for (int pc : *pcts) marks[i].push_back(std::max(0, (nets[i]->n_leaves() - 1) * std::min(std::max(pc, 0), 100) / 100));
      std::sort(marks[i].begin(), marks[i].end());
      marks[i].erase(std::unique(marks[i].begin(), marks[i].end()), marks[i].end());
    }
  auto take_snaps = [&](int i) {  // snapshot at every checkpoint reached; true once past the last
    while (!marks[i].empty() && snaps[i].size() < marks[i].size() && merged[i] >= marks[i][snaps[i].size()])
      snaps[i].push_back(st[i]);
    return !marks[i].empty() && snaps[i].size() == marks[i].size();
  };
  if (chosen) chosen->assign(n, {});
  std::vector<std::vector<Cand>> cs(n);
  std::vector<float> X, Y;
  const size_t max_rows = (size_t)n * cands;
  if (d_params_bf16 && ws_bytes < max_rows * (TNC_MLP_FEATURES + 1) * sizeof(float))
    return set_error(TNC_ERR_BUFFER, "learned planning workspace too small");
  float* dX = (float*)d_ws;
  float* dY = dX + max_rows * TNC_MLP_FEATURES;
  for (;;) {
    X.clear();
    std::vector<std::pair<int, int>> span(n, {0, 0});
    for (int i = 0; i < n; i++) {
      if (take_snaps(i)) {  // coarsening done for this formula
        cs[i].clear();
        continue;
      }
      top_candidates(st[i], cs[i], d_params_bf16 ? cands : 1);
      span[i] = {(int)(X.size() / TNC_MLP_FEATURES), (int)cs[i].size()};
      const int lm = cs[i].empty() ? 0 : live_max_rank(st[i]);
      for (size_t c = 0; c < cs[i].size(); c++) {
        float f[TNC_MLP_FEATURES];
        features(st[i], cs[i][c], lm, (int)c, (int)cs[i].size(), f);
        X.insert(X.end(), f, f + TNC_MLP_FEATURES);
      }
    }
    const int64_t rows = (int64_t)(X.size() / TNC_MLP_FEATURES);
    if (rows == 0) break;
    Y.assign(rows, 0.f);
    if (d_params_bf16) {
      int rc = TNC_OK;
      copy_device(dX, X.data(), X.size() * sizeof(float), 0, stream, &rc);
      if (rc) return rc;
      rc = mlp_forward_bf16_dev(d_params_bf16, dX, rows, dY, stream);
      if (rc) return rc;
      copy_device(Y.data(), dY, rows * sizeof(float), 1, stream, &rc);
      if (rc) return rc;
    }
    for (int i = 0; i < n; i++) {
      if (span[i].second == 0) continue;
      int best = 0;
      for (int c = 1; c < span[i].second; c++)
        if (Y[span[i].first + c] < Y[span[i].first + best]) best = c;
      if (chosen) (*chosen)[i].push_back(best);
      st[i].merge(cs[i][best].a, cs[i][best].b);
      merged[i]++;
    }
  }
  trees.resize(n);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < n; i++) {
    if (completion && !snaps[i].empty()) {  // finish every snapshot by the heuristic, keep the cheapest
      int best = -1;
      TreeCost bc;
      for (size_t j = 0; j < snaps[i].size(); j++) {
        complete_with(snaps[i][j], *nets[i], *completion);
        const TreeCost c = tree_cost(snaps[i][j].t);
        if (best < 0 || cheaper_cost(c, bc)) {
          best = (int)j;
          bc = c;
        }
      }
      trees[i] = std::move(snaps[i][best].t);
      continue;
    }
    st[i].finish_greedy();  // joins disconnected leftovers
    trees[i] = std::move(st[i].t);
  }
  return TNC_OK;
}

// TNC_PLAN_COARSEN: the paper's heuristics (Sec. 3.1.1) used at two levels.
// Tensor-greedy merges coarsen the network; at 10, 20, ..., 80 % of its
// merges the network of the live tensors is finished by TNC_PLAN_BEST (the
// coarse leaves are the live tensors, Sec. 2.2).  These plans, and
// tensor-greedy, tensor-METIS and tensor-GN on the whole network, are the
// candidates; their exact costs are known before any contraction (the lazy
// evaluation of Sec. 4).  Kept: the fewest MACs among the candidates within the
// rank cap (ties: smaller max rank); if none fits, the smallest (max rank, MACs).
int plan_coarsen(const Network& net, const tnc_plan_opts& o, Tree& out) {
  if (net.n_leaves() < 2) return plan_greedy(net, out);
  std::vector<Tree> cands(3);
  int rc = plan_greedy(net, cands[0]);
  if (rc == TNC_OK) rc = plan_bisect(net, o.tries > 0 ? o.tries : 2, o.seed, cands[1]);
  if (rc == TNC_OK) rc = plan_gn(net, cands[2]);
  if (rc != TNC_OK) return rc;
  GState s;
  s.init(net);
  std::vector<int> marks;
  for (int pc = 10; pc <= 80; pc += 10) marks.push_back((net.n_leaves() - 1) * pc / 100);
  marks.erase(std::unique(marks.begin(), marks.end()), marks.end());
  std::vector<GState> snaps;
  std::vector<Cand> cs;
  for (int merged = 0; snaps.size() < marks.size();) {
    while (snaps.size() < marks.size() && merged >= marks[snaps.size()]) snaps.push_back(s);
    if (snaps.size() == marks.size()) break;
    top_candidates(s, cs, 1);
    if (cs.empty()) break;  // no two live tensors share a bond: coarsening ends here
    s.merge(cs[0].a, cs[0].b);
    merged++;
  }
  tnc_plan_opts best{};
  best.heuristic = TNC_PLAN_BEST;
  best.tries = o.tries;
  best.seed = o.seed;
  for (GState& g : snaps) {
    complete_with(g, net, best);
    cands.push_back(std::move(g.t));
  }
  const int cap = o.rank_cap > 0 ? o.rank_cap : 32;
  int pick = -1;
  TreeCost pc{};
  for (size_t i = 0; i < cands.size(); i++) {
    const TreeCost c = tree_cost(cands[i]);
    bool better;
    if (pick < 0) better = true;
    else if ((c.max_rank <= cap) != (pc.max_rank <= cap)) better = c.max_rank <= cap;
    else if (c.max_rank <= cap) better = c.macs < pc.macs || (c.macs == pc.macs && c.max_rank < pc.max_rank);
    else better = cheaper_cost(c, pc);
    if (better) {
      pick = (int)i;
      pc = c;
    }
  }
  out = std::move(cands[pick]);
  return TNC_OK;
}

}  // namespace tnc

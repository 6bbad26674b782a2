// Bond slicing behind the C ABI: the choice of the variables to fix, the
// restricted networks of the slices and their plans.
//
// Fixing variable v to x splits the full trace of the network (Eq. z,
// Sec. 2.1) into the traces with x_v = 0 and x_v = 1: v's COPY tensor leaves
// the network and every clause tensor on one of its bonds is restricted to the
// fixed value (it becomes a table over its remaining bonds).  No tensor grows;
// the memory of the contraction, which the paper names as the bottleneck of
// its method (Sec. 4), shrinks, at the price of 2^s contractions whose counts
// are added.
//
// All slices of one set of fixed variables have the same network structure
// (the same tensors and bonds; only table entries differ), so one plan serves
// them all.  Each round adds the variable whose slices have the cheapest exact
// plan cost (the lazy evaluation of Sec. 4: smallest max rank, then fewest
// MACs in all), preferring variables whose slices need no more MACs in all
// than the current ones.  Every candidate is planned afresh by the caller's heuristic
// and also by the current plan restricted to the slice (the same tree with the
// fixed variable's tensor left out); the cheaper is kept, so the max rank
// never grows from one round to the next.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tnc_internal.h"

namespace tnc {

int finish_plan(tnc_plan_t* p, int rank_cap, tnc_plan_stats* stats);

namespace {

// A formula in host vectors (the network's own description of it).
struct FormulaV {
  int n_vars = 0;
  std::vector<std::vector<int>> clauses;
  std::vector<uint8_t> kinds;
  std::vector<std::vector<uint32_t>> tables;  // TABLE clauses only
  std::vector<int> open_vars;
};

// The formula a network was built from: clause c's variables are the var
// leaves at the far end of its bonds, in bond order.
FormulaV formula_of(const Network& net) {
  FormulaV f;
  f.n_vars = net.n_vars;
  f.open_vars = net.open_vars;
  const int m = net.n_cons;
  for (int c = 0; c < m; c++) {
    const Leaf& L = net.leaves[c];
    std::vector<int> vs;
    for (int b : L.bonds) vs.push_back(net.bond_end1[b] - m);
    f.clauses.push_back(vs);
    f.kinds.push_back(L.kind);
    f.tables.push_back(L.kind == LK_TABLE ? L.table : std::vector<uint32_t>());
  }
  return f;
}

// Entry idx (bit j = value of the clause's j-th variable) of a clause tensor:
// exactly one (Eq. 1in3), OR (Eq. or), NAND, or the table.
uint32_t clause_entry(uint8_t kind, int d, uint32_t idx, const std::vector<uint32_t>& table) {
  switch (kind) {
    case LK_1IN3: return __builtin_popcount(idx) == 1 ? 1u : 0u;
    case LK_OR: return idx != 0 ? 1u : 0u;
    case LK_NAND: return idx != ((1u << d) - 1u) ? 1u : 0u;
    default: return table[idx];
  }
}

// The formula with vars[i] fixed to bit i of `bits`: fixed variables leave
// (the others are renumbered in order, new_id[v] = -1 for fixed ones) and a
// clause on a fixed variable becomes the TABLE over its remaining variables.
FormulaV slice_formula(const FormulaV& f, const std::vector<int>& vars, uint32_t bits, std::vector<int>& new_id) {
  std::vector<int> val(f.n_vars, -1);
  for (size_t i = 0; i < vars.size(); i++) val[vars[i]] = (int)((bits >> i) & 1u);
  new_id.assign(f.n_vars, -1);
  FormulaV g;
  for (int v = 0; v < f.n_vars; v++)
    if (val[v] < 0) new_id[v] = g.n_vars++;
  for (int v : f.open_vars) g.open_vars.push_back(new_id[v]);
  for (size_t c = 0; c < f.clauses.size(); c++) {
    const std::vector<int>& cl = f.clauses[c];
    const int d = (int)cl.size();
    std::vector<int> free_pos;
    uint32_t base = 0;
    for (int j = 0; j < d; j++) {
      if (val[cl[j]] < 0) free_pos.push_back(j);
      else base |= (uint32_t)val[cl[j]] << j;
    }
    std::vector<int> ncl;
    for (int j : free_pos) ncl.push_back(new_id[cl[j]]);
    g.clauses.push_back(ncl);
    if ((int)free_pos.size() == d) {
      g.kinds.push_back(f.kinds[c]);
      g.tables.push_back(f.tables[c]);
      continue;
    }
    std::vector<uint32_t> tab((size_t)1 << free_pos.size());
    for (uint32_t i = 0; i < tab.size(); i++) {
      uint32_t idx = base;
      for (size_t q = 0; q < free_pos.size(); q++) idx |= ((i >> q) & 1u) << free_pos[q];
      tab[i] = clause_entry(f.kinds[c], d, idx, f.tables[c]);
    }
    g.kinds.push_back(LK_TABLE);
    g.tables.push_back(std::move(tab));
  }
  return g;
}

int network_of(const FormulaV& f, Network& out) {
  std::vector<int32_t> arity, var_of, open(f.open_vars.begin(), f.open_vars.end());
  std::vector<uint32_t> table;
  for (size_t c = 0; c < f.clauses.size(); c++) {
    arity.push_back((int32_t)f.clauses[c].size());
    for (int v : f.clauses[c]) var_of.push_back(v);
    if (f.kinds[c] == LK_TABLE) table.insert(table.end(), f.tables[c].begin(), f.tables[c].end());
  }
  tnc_formula tf;
  tf.n_vars = f.n_vars;
  tf.n_cons = (int32_t)f.clauses.size();
  tf.arity = arity.data();
  tf.var_of = var_of.data();
  tf.kind = f.kinds.data();
  tf.table = table.data();
  tf.n_open = (int32_t)open.size();
  tf.open_vars = open.data();
  return build_network(&tf, out);
}

bool cheaper(const TreeCost& a, const TreeCost& b) {
  return a.max_rank != b.max_rank ? a.max_rank < b.max_rank : a.macs < b.macs;
}

// The tree `t` of the network of fixed set F restricted to the network of
// F + {v}: leaf map from the first network's leaf ids to the second's (-1:
// the fixed variable's tensor, left out); every merge with a left-out side
// disappears.
void restrict_tree(const Tree& t, const std::vector<int>& leaf_map, const Network& net2, Tree& out) {
  std::vector<int> id(t.nodes.size(), -1);
  for (int i = 0; i < t.n_leaves; i++) id[i] = leaf_map[i];
  std::vector<std::pair<int, int>> merges;
  const int L2 = net2.n_leaves();
  for (size_t i = t.n_leaves; i < t.nodes.size(); i++) {
    const int a = id[t.nodes[i].left], b = id[t.nodes[i].right];
    if (a < 0) id[i] = b;
    else if (b < 0) id[i] = a;
    else {
      merges.push_back({a, b});
      id[i] = L2 + (int)merges.size() - 1;
    }
  }
  tree_from_merges(net2, merges, out);
}

struct Candidate {
  int var = -1;
  Tree tree;
  TreeCost cost;
  bool ok = false;
};

}  // namespace

// Chooses s variables and plans the 2^s slices (see tnc.h).
int plan_sliced(const Network& net, int s, const tnc_plan_opts& opts, std::vector<tnc_plan_t*>& out,
                std::vector<int>& vars, std::vector<tnc_plan_stats>& stats) {
  const FormulaV f = formula_of(net);
  std::vector<char> is_open(f.n_vars, 0);
  for (int v : f.open_vars) is_open[v] = 1;
  vars.clear();
  // the current representative slice (fixed variables all 0) and its plan
  Network cur_net = net;
  std::vector<int> cur_id(f.n_vars);
  for (int v = 0; v < f.n_vars; v++) cur_id[v] = v;
  Tree cur_tree;
  int rc = plan_tree(cur_net, opts, cur_tree);
  if (rc) return rc;
  TreeCost cur_cost = tree_cost(cur_tree);
  for (int round = 0; round < s; round++) {
    // candidates: the variables on the tensors of largest rank (most such
    // bonds first), not open, not fixed
    std::vector<int> score(f.n_vars, 0);
    const int m = cur_net.n_cons;
    std::vector<int> orig(cur_net.n_vars, -1);
    for (int v = 0; v < f.n_vars; v++)
      if (cur_id[v] >= 0) orig[cur_id[v]] = v;
    for (const Node& nd : cur_tree.nodes) {
      if ((int)nd.bonds.size() < cur_cost.max_rank) continue;
      for (int b : nd.bonds) {
        const int e = cur_net.bond_end1[b];
        if (e < m) continue;  // an open bond
        const int v = orig[e - m];
        if (!is_open[v]) score[v]++;
      }
    }
    std::vector<int> cand;
    for (int v = 0; v < f.n_vars; v++)
      if (score[v] > 0) cand.push_back(v);
    if (cand.empty())
      for (int v = 0; v < f.n_vars; v++)
        if (cur_id[v] >= 0 && !is_open[v]) cand.push_back(v);
    if (cand.empty()) return set_error(TNC_ERR_INVALID, "no variable left to slice");
    std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) { return score[a] > score[b]; });
    if (cand.size() > 48) cand.resize(48);
    std::vector<Candidate> res(cand.size());
    int fail_rc = TNC_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int ci = 0; ci < (int)cand.size(); ci++) {
      Candidate& C = res[ci];
      C.var = cand[ci];
      std::vector<int> fixed = vars;
      fixed.push_back(C.var);
      std::vector<int> nid;
      const FormulaV g = slice_formula(f, fixed, 0u, nid);
      Network gn;
      if (network_of(g, gn) != TNC_OK) {
#pragma omp critical
        fail_rc = TNC_ERR_INVALID;
        continue;
      }
      Tree fresh;
      if (plan_tree(gn, opts, fresh) != TNC_OK) continue;
      // the current plan, restricted: clause leaves keep their ids; variable
      // leaves move to the new numbering
      std::vector<int> leaf_map(cur_net.n_leaves(), -1);
      for (int c = 0; c < m; c++) leaf_map[c] = c;
      for (int v = 0; v < f.n_vars; v++)
        if (cur_id[v] >= 0 && nid[v] >= 0) leaf_map[m + cur_id[v]] = m + nid[v];
      Tree inh;
      restrict_tree(cur_tree, leaf_map, gn, inh);
      const TreeCost cf = tree_cost(fresh), ci2 = tree_cost(inh);
      if (cheaper(ci2, cf)) {
        C.tree = std::move(inh);
        C.cost = ci2;
      } else {
        C.tree = std::move(fresh);
        C.cost = cf;
      }
      C.ok = true;
    }
    if (fail_rc) return set_error(fail_rc, "slice network could not be built");
    // among the candidates whose slices need no more MACs in all than the
    // current slices (twice as many slices, so at most half the MACs each),
    // the cheapest; if there is none, the cheapest of all
    int best = -1, best_any = -1;
    for (size_t i = 0; i < res.size(); i++) {
      if (!res[i].ok) continue;
      if (best_any < 0 || cheaper(res[i].cost, res[best_any].cost)) best_any = (int)i;
      if (2.0 * res[i].cost.macs <= cur_cost.macs && (best < 0 || cheaper(res[i].cost, res[best].cost)))
        best = (int)i;
    }
    if (best < 0) best = best_any;
    if (best < 0) return set_error(TNC_ERR_INVALID, "no slice could be planned");
    vars.push_back(res[best].var);
    std::vector<int> nid;
    const FormulaV g = slice_formula(f, vars, 0u, nid);
    rc = network_of(g, cur_net);
    if (rc) return rc;
    cur_id = nid;
    cur_tree = std::move(res[best].tree);
    cur_cost = res[best].cost;
  }
  // every slice: its own network (tables differ), the representative's tree
  const size_t n = (size_t)1 << vars.size();
  out.assign(n, nullptr);
  stats.assign(n, tnc_plan_stats{});
  for (size_t j = 0; j < n; j++) {
    std::vector<int> nid;
    const FormulaV g = slice_formula(f, vars, (uint32_t)j, nid);
    auto* p = new tnc_plan_t();
    rc = network_of(g, p->net);
    if (!rc) {
      p->tree = cur_tree;
      rc = finish_plan(p, opts.rank_cap, &stats[j]);
    }
    if (rc) {
      delete p;
      for (tnc_plan_t*& q : out) {
        delete q;
        q = nullptr;
      }
      return rc;
    }
    out[j] = p;
  }
  return TNC_OK;
}

}  // namespace tnc

extern "C" int tnc_slice_network(const tnc_network_t* net, int32_t s, const int32_t* vars, uint32_t bits,
                                 tnc_network_t** out) {
  using namespace tnc;
  clear_error();
  if (!net || !out || s < 0 || s > 31 || (s > 0 && !vars)) return set_error(TNC_ERR_INVALID, "bad arguments");
  *out = nullptr;
  try {
    const FormulaV f = formula_of(net->net);
    std::vector<int> vs(vars, vars + s), nid;
    std::vector<char> seen(f.n_vars, 0);
    for (int v : vs) {
      if (v < 0 || v >= f.n_vars || seen[v]) return set_error(TNC_ERR_INVALID, "bad or repeated variable");
      seen[v] = 1;
    }
    for (int v : f.open_vars)
      if (seen[v]) return set_error(TNC_ERR_INVALID, "open variables cannot be sliced");
    auto* h = new tnc_network_t();
    const int rc = network_of(slice_formula(f, vs, bits, nid), h->net);
    if (rc) {
      delete h;
      return rc;
    }
    *out = h;
    return TNC_OK;
  } catch (const std::bad_alloc&) {
    return set_error(TNC_ERR_NOMEM, "out of host memory");
  }
}

extern "C" int tnc_network_formula(const tnc_network_t* net, int32_t* n_vars, int32_t* n_cons, int32_t* n_occ,
                                   int32_t* n_table, int32_t* n_open, int32_t* arity, int32_t* var_of, uint8_t* kind,
                                   uint32_t* table, int32_t* open_vars) {
  using namespace tnc;
  clear_error();
  if (!net) return set_error(TNC_ERR_INVALID, "network is NULL");
  const FormulaV f = formula_of(net->net);
  int32_t occ = 0, tab = 0;
  for (size_t c = 0; c < f.clauses.size(); c++) {
    if (arity) arity[c] = (int32_t)f.clauses[c].size();
    if (kind) kind[c] = f.kinds[c];
    for (int v : f.clauses[c]) {
      if (var_of) var_of[occ] = v;
      occ++;
    }
    if (f.kinds[c] == LK_TABLE)
      for (uint32_t w : f.tables[c]) {
        if (table) table[tab] = w;
        tab++;
      }
  }
  for (size_t i = 0; i < f.open_vars.size(); i++)
    if (open_vars) open_vars[i] = f.open_vars[i];
  if (n_vars) *n_vars = f.n_vars;
  if (n_cons) *n_cons = (int32_t)f.clauses.size();
  if (n_occ) *n_occ = occ;
  if (n_table) *n_table = tab;
  if (n_open) *n_open = (int32_t)f.open_vars.size();
  return TNC_OK;
}

extern "C" int tnc_plan_sliced(const tnc_network_t* net, int32_t s, const tnc_plan_opts* opts, tnc_plan_t** out,
                               int32_t* vars_out, tnc_plan_stats* stats) {
  using namespace tnc;
  clear_error();
  if (!net || !opts || !out || (s > 0 && !vars_out)) return set_error(TNC_ERR_INVALID, "NULL argument");
  if (s < 0 || s > 16) return set_error(TNC_ERR_INVALID, "s must be in [0, 16]");
  try {
    std::vector<tnc_plan_t*> plans;
    std::vector<int> vars;
    std::vector<tnc_plan_stats> st;
    const int rc = plan_sliced(net->net, s, *opts, plans, vars, st);
    if (rc) return rc;
    for (size_t j = 0; j < plans.size(); j++) {
      out[j] = plans[j];
      if (stats) stats[j] = st[j];
    }
    for (int i = 0; i < s; i++) vars_out[i] = vars[i];
    return TNC_OK;
  } catch (const std::bad_alloc&) {
    return set_error(TNC_ERR_NOMEM, "out of host memory");
  }
}

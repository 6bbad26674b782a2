// C ABI, host-only half: library info, networks and plans.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "tnc_internal.h"

namespace tnc {
const char* last_error_cstr();
}

using namespace tnc;

extern "C" {

const char* tnc_version(void) { return "tnc 0.1 (sm_103a)"; }

const char* tnc_last_error(void) { return last_error_cstr(); }

int tnc_default_primes(int32_t n, uint32_t* out) {
  clear_error();
  if (n < 0 || n > 64 || (n > 0 && !out)) return set_error(TNC_ERR_INVALID, "n must be in [0, 64]");
  std::vector<uint32_t> p = default_primes(n);
  std::copy(p.begin(), p.end(), out);
  return TNC_OK;
}

int tnc_build_network(const tnc_formula* f, tnc_network_t** out) {
  clear_error();
  if (!out) return set_error(TNC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  try {
    auto* h = new tnc_network_t();
    int rc = build_network(f, h->net);
    if (rc != TNC_OK) {
      delete h;
      return rc;
    }
    *out = h;
    return TNC_OK;
  } catch (const std::bad_alloc&) {
    return set_error(TNC_ERR_NOMEM, "out of host memory");
  } catch (...) {
    return set_error(TNC_ERR_INVALID, "unexpected failure in tnc_build_network");
  }
}

int tnc_network_info(const tnc_network_t* net, int32_t* n_tensors, int32_t* n_bonds, int32_t* n_components) {
  clear_error();
  if (!net) return set_error(TNC_ERR_INVALID, "network is NULL");
  if (n_tensors) *n_tensors = net->net.n_leaves();
  if (n_bonds) *n_bonds = net->net.n_bonds;
  if (n_components) *n_components = net->net.n_components;
  return TNC_OK;
}

void tnc_free_network(tnc_network_t* net) { delete net; }

int tnc_plan(const tnc_network_t* net, const tnc_plan_opts* opts, tnc_plan_t** out, tnc_plan_stats* stats) {
  clear_error();
  if (!net || !opts || !out) return set_error(TNC_ERR_INVALID, "NULL argument");
  *out = nullptr;
  try {
    auto* p = new tnc_plan_t();
    p->net = net->net;
    int rc = plan_tree(p->net, *opts, p->tree);
    if (rc == TNC_OK) {
      p->cost = tree_cost(p->tree);
      const int cap = opts->rank_cap > 0 ? opts->rank_cap : 32;
      if (p->cost.max_rank > cap)
        rc = set_error(TNC_ERR_TOO_LARGE, "plan rank " + std::to_string(p->cost.max_rank) +
                                              " exceeds rank cap " + std::to_string(cap));
    }
    if (rc == TNC_OK) rc = lower_plan(p->net, p->tree, p->low);
    if (rc == TNC_OK) rc = validate_lowered(p->net, p->tree, p->low);
    if (rc != TNC_OK) {
      if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->max_rank = p->cost.max_rank;
      }
      delete p;
      return rc;
    }
    tnc_plan_stats& s = p->stats;
    s.max_rank = p->cost.max_rank;
    s.n_steps = (int32_t)p->tree.nodes.size() - p->tree.n_leaves;
    s.n_leaves = p->tree.n_leaves;
    s.depth = p->cost.depth;
    s.total_macs = p->cost.macs;
    s.total_entries = p->cost.entries;
    s.log2_bound = p->net.log2_bound;
    s.arena_entries = p->low.seq_arena_entries;
    s.batch_arena_entries = p->low.lvl_arena_entries;
    s.n_dense_steps = 0;
    s.dense_macs = 0;
    for (const StepDesc& d : p->low.seq_steps)
      if (tc_eligible(d)) {
        s.n_dense_steps++;
        s.dense_macs += std::ldexp(1.0, d.ka + d.kb + d.k);
      }
    if (stats) *stats = s;
    *out = p;
    return TNC_OK;
  } catch (const std::bad_alloc&) {
    return set_error(TNC_ERR_NOMEM, "out of host memory");
  } catch (...) {
    return set_error(TNC_ERR_INVALID, "unexpected failure in tnc_plan");
  }
}

int tnc_plan_many(const tnc_network_t* const* nets, int32_t n, const tnc_plan_opts* opts, tnc_plan_t** out,
                  tnc_plan_stats* stats) {
  clear_error();
  if (!nets || n < 0 || !opts || !out) return set_error(TNC_ERR_INVALID, "NULL argument");
  int first_rc = TNC_OK;
  std::string first_msg;
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < n; i++) {
    tnc_plan_t* p = nullptr;
    tnc_plan_stats st{};
    int rc = tnc_plan(nets[i], opts, &p, &st);
    out[i] = p;
    if (stats) stats[i] = st;
    if (rc != TNC_OK) {
#pragma omp critical
      {
        if (first_rc == TNC_OK) {
          first_rc = rc;
          first_msg = "formula " + std::to_string(i) + ": " + tnc_last_error();
        }
      }
    }
  }
  if (first_rc != TNC_OK) {
    for (int i = 0; i < n; i++) {
      tnc_free_plan(out[i]);
      out[i] = nullptr;
    }
    return set_error(first_rc, first_msg);
  }
  return TNC_OK;
}

int tnc_plan_steps(const tnc_plan_t* plan, int32_t* left, int32_t* right, int32_t cap) {
  clear_error();
  if (!plan) return set_error(TNC_ERR_INVALID, "plan is NULL");
  const int n = (int)plan->tree.nodes.size() - plan->tree.n_leaves;
  if (cap < n || (n > 0 && (!left || !right))) return set_error(TNC_ERR_BUFFER, "need " + std::to_string(n) + " entries");
  for (int i = 0; i < n; i++) {
    left[i] = plan->tree.nodes[plan->tree.n_leaves + i].left;
    right[i] = plan->tree.nodes[plan->tree.n_leaves + i].right;
  }
  return TNC_OK;
}

void tnc_free_plan(tnc_plan_t* plan) { delete plan; }

}  // extern "C"

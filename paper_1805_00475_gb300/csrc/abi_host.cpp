// C ABI, host-only half: library info, networks and plans.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "tnc_internal.h"

namespace tnc {
const char* last_error_cstr();
}

using namespace tnc;

namespace tnc {

// Cost, rank cap, lowering, validation and stats of a plan whose tree is set.
int finish_plan(tnc_plan_t* p, int rank_cap, tnc_plan_stats* stats) {
  p->cost = tree_cost(p->tree);
  const int cap = rank_cap > 0 ? rank_cap : 32;
  int rc = TNC_OK;
  if (p->cost.max_rank > cap)
    rc = set_error(TNC_ERR_TOO_LARGE, "plan rank " + std::to_string(p->cost.max_rank) + " exceeds rank cap " +
                                          std::to_string(cap));
  if (rc == TNC_OK) rc = lower_plan(p->net, p->tree, p->low);
  if (rc == TNC_OK) rc = validate_lowered(p->net, p->tree, p->low);
  if (rc != TNC_OK) {
    if (stats) {
      std::memset(stats, 0, sizeof(*stats));
      stats->max_rank = p->cost.max_rank;
      stats->total_macs = p->cost.macs;
    }
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
  s.n_dense_steps_p8 = 0;
  s.dense_macs_p8 = 0;
  for (const StepDesc& d : p->low.seq_steps) {
    if (tc_eligible(d)) {
      s.n_dense_steps++;
      s.dense_macs += std::ldexp(1.0, d.ka + d.kb + d.k);
    }
    if (p8_eligible(d)) {
      s.n_dense_steps_p8++;
      s.dense_macs_p8 += std::ldexp(1.0, d.ka + d.kb + d.k);
    }
  }
  s.n_direct_p8 = 0;
  for (uint8_t x : p->low.p8_direct) s.n_direct_p8 += x;
  s.p8_arena_entries = p->low.p8_arena_entries;
  if (stats) *stats = s;
  return TNC_OK;
}

int learned_dataset(const std::vector<const Network*>& nets, int states, int cands, uint64_t seed, std::vector<float>& X,
                    std::vector<float>& T, const std::vector<std::vector<int>>* policy,
                    const tnc_plan_opts* completion, int max_pct);
int learned_trees(const std::vector<const Network*>& nets, const void* d_params_bf16, void* d_ws, size_t ws_bytes,
                  void* stream, int cands, std::vector<Tree>& trees, std::vector<std::vector<int>>* chosen,
                  const tnc_plan_opts* completion, const std::vector<int>* pcts);

}  // namespace tnc

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

int tnc_default_primes_p8(int32_t n, uint32_t* out) {
  clear_error();
  if (n < 0 || n > kP8MaxResidues || (n > 0 && !out)) return set_error(TNC_ERR_INVALID, "n must be in [0, 53]");
  std::vector<uint32_t> p = default_primes_p8(n);
  std::copy(p.begin(), p.end(), out);
  return TNC_OK;
}

int tnc_build_network(const tnc_formula* f, tnc_network_t** out) {
  clear_error();
  if (!out) return set_error(TNC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  try {
    if (inject_hit(TNC_INJECT_NOMEM)) throw std::bad_alloc();
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
    if (inject_hit(TNC_INJECT_NOMEM)) throw std::bad_alloc();
    auto* p = new tnc_plan_t();
    p->net = net->net;
    int rc = plan_tree(p->net, *opts, p->tree);
    if (rc == TNC_OK && inject_hit(TNC_INJECT_PLAN))
      rc = set_error(TNC_ERR_TOO_LARGE, "injected failure (TNC_INJECT_PLAN)");
    if (rc == TNC_OK) rc = finish_plan(p, opts->rank_cap, stats);
    if (rc != TNC_OK) {
      delete p;
      return rc;
    }
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

// Scorer parameter files: "TNCMLP01", then u32 features, hidden width and
// parameter count, the fp32 parameters, and a 64-bit FNV-1a checksum of all
// the bytes before it (little-endian throughout).
static uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t h = 0xCBF29CE484222325ull) {
  for (size_t i = 0; i < n; i++) {
    h ^= p[i];
    h *= 0x100000001B3ull;
  }
  return h;
}

int tnc_learned_save(const char* path, const float* params) {
  clear_error();
  if (!path || !params) return set_error(TNC_ERR_INVALID, "NULL argument");
  std::vector<unsigned char> buf(8 + 12 + sizeof(float) * TNC_MLP_PARAMS);
  std::memcpy(buf.data(), "TNCMLP01", 8);
  const uint32_t hdr[3] = {TNC_MLP_FEATURES, TNC_MLP_HIDDEN, TNC_MLP_PARAMS};
  std::memcpy(buf.data() + 8, hdr, 12);
  std::memcpy(buf.data() + 20, params, sizeof(float) * TNC_MLP_PARAMS);
  const uint64_t sum = fnv1a(buf.data(), buf.size());
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return set_error(TNC_ERR_INVALID, std::string("cannot open ") + path + " for writing");
  const bool ok = std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size() && std::fwrite(&sum, 8, 1, fp) == 1;
  if (std::fclose(fp) != 0 || !ok) return set_error(TNC_ERR_INVALID, std::string("write failed: ") + path);
  return TNC_OK;
}

int tnc_learned_load(const char* path, float* params) {
  clear_error();
  if (!path || !params) return set_error(TNC_ERR_INVALID, "NULL argument");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return set_error(TNC_ERR_INVALID, std::string("cannot open ") + path);
  std::vector<unsigned char> buf(8 + 12 + sizeof(float) * TNC_MLP_PARAMS);
  uint64_t sum = 0;
  const bool ok = std::fread(buf.data(), 1, buf.size(), fp) == buf.size() && std::fread(&sum, 8, 1, fp) == 1 &&
                  std::fgetc(fp) == EOF;
  std::fclose(fp);
  if (!ok) return set_error(TNC_ERR_INVALID, std::string("truncated or oversized parameter file: ") + path);
  uint32_t hdr[3];
  std::memcpy(hdr, buf.data() + 8, 12);
  if (std::memcmp(buf.data(), "TNCMLP01", 8) != 0 || hdr[0] != TNC_MLP_FEATURES || hdr[1] != TNC_MLP_HIDDEN ||
      hdr[2] != TNC_MLP_PARAMS)
    return set_error(TNC_ERR_INVALID, "not a scorer parameter file of this layout");
  if (fnv1a(buf.data(), buf.size()) != sum) return set_error(TNC_ERR_INVALID, "parameter file checksum mismatch");
  std::memcpy(params, buf.data() + 20, sizeof(float) * TNC_MLP_PARAMS);
  return TNC_OK;
}

int tnc_mlp_init(uint64_t seed, float* params) {
  clear_error();
  if (!params) return set_error(TNC_ERR_INVALID, "params is NULL");
  const int F = TNC_MLP_FEATURES, H = TNC_MLP_HIDDEN;
  uint64_t st = seed;
  auto u01 = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  auto normal = [&]() { return std::sqrt(-2.0 * std::log(u01())) * std::cos(6.283185307179586 * u01()); };
  float* p = params;
  for (int i = 0; i < F * H; i++) *p++ = (float)(normal() * std::sqrt(2.0 / F));  // W1
  for (int i = 0; i < H; i++) *p++ = 0.f;                                       // b1
  for (int i = 0; i < H * H; i++) *p++ = (float)(normal() * std::sqrt(2.0 / H));  // W2
  for (int i = 0; i < H; i++) *p++ = 0.f;                                       // b2
  for (int i = 0; i < H; i++) *p++ = (float)(normal() * std::sqrt(1.0 / H));    // w3
  *p++ = 0.f;                                                                   // b3
  return TNC_OK;
}

int tnc_learned_dataset(const tnc_network_t* const* nets, int32_t n, int32_t states, int32_t cands, uint64_t seed,
                        float* x, float* t, int64_t cap_rows, int64_t* n_rows) {
  clear_error();
  if (!nets || n < 0 || states <= 0 || cands <= 1 || !n_rows) return set_error(TNC_ERR_INVALID, "bad dataset arguments");
  try {
    std::vector<const Network*> v;
    for (int i = 0; i < n; i++) {
      if (!nets[i]) return set_error(TNC_ERR_INVALID, "NULL network");
      v.push_back(&nets[i]->net);
    }
    std::vector<float> X, T;
    learned_dataset(v, states, cands, seed, X, T, nullptr, nullptr, 100);
    *n_rows = (int64_t)T.size();
    if (!x || !t || cap_rows < (int64_t)T.size())
      return set_error(TNC_ERR_BUFFER, "need " + std::to_string(T.size()) + " rows");
    std::copy(X.begin(), X.end(), x);
    std::copy(T.begin(), T.end(), t);
    return TNC_OK;
  } catch (const std::bad_alloc&) {
    return set_error(TNC_ERR_NOMEM, "out of host memory");
  }
}

int tnc_learned_dataset_on_policy(const tnc_network_t* const* nets, int32_t n, const void* d_params_bf16,
                                  void* d_ws, size_t ws_bytes, void* cuda_stream, int32_t states, uint64_t seed,
                                  float* x, float* t, int64_t cap_rows, int64_t* n_rows) {
  clear_error();
  if (!nets || n <= 0 || !d_params_bf16 || !d_ws || states <= 0 || !n_rows)
    return set_error(TNC_ERR_INVALID, "bad dataset arguments");
  try {
    std::vector<const Network*> v;
    for (int i = 0; i < n; i++) {
      if (!nets[i]) return set_error(TNC_ERR_INVALID, "NULL network");
      v.push_back(&nets[i]->net);
    }
    std::vector<Tree> trees;
    std::vector<std::vector<int>> chosen;
    int rc = learned_trees(v, d_params_bf16, d_ws, ws_bytes, cuda_stream, TNC_LEARNED_CANDIDATES, trees, &chosen,
                           nullptr, nullptr);
    if (rc) return rc;
    std::vector<float> X, T;
    learned_dataset(v, states, TNC_LEARNED_CANDIDATES, seed, X, T, &chosen, nullptr, 100);
    *n_rows = (int64_t)T.size();
    if (!x || !t || cap_rows < (int64_t)T.size())
      return set_error(TNC_ERR_BUFFER, "need " + std::to_string(T.size()) + " rows");
    std::copy(X.begin(), X.end(), x);
    std::copy(T.begin(), T.end(), t);
    return TNC_OK;
  } catch (const std::bad_alloc&) {
    return set_error(TNC_ERR_NOMEM, "out of host memory");
  }
}

size_t tnc_plan_learned_workspace_bytes(int32_t n) {
  return n <= 0 ? 0 : (size_t)n * TNC_LEARNED_CANDIDATES * (TNC_MLP_FEATURES + 1) * sizeof(float);
}

static int plan_learned_impl(const tnc_network_t* const* nets, int32_t n, const void* d_params_bf16,
                             const tnc_learned_opts* lo, const tnc_plan_opts* fallback, void* d_ws, size_t ws_bytes,
                             void* cuda_stream, tnc_plan_t** out, tnc_plan_stats* stats, int32_t* chose_learned,
                             double* learned_macs) {
  if (!nets || n <= 0 || (!lo && !d_params_bf16) || (d_params_bf16 && !d_ws) || !out)
    return set_error(TNC_ERR_INVALID, "bad arguments");
  for (int i = 0; i < n; i++) out[i] = nullptr;
  try {
    std::vector<const Network*> v;
    for (int i = 0; i < n; i++) {
      if (!nets[i]) return set_error(TNC_ERR_INVALID, "NULL network");
      v.push_back(&nets[i]->net);
    }
    std::vector<Tree> trees;
    tnc_plan_opts comp{};
    std::vector<int> pcts;
    if (lo) {
      comp.heuristic = lo->completion;
      comp.tries = 2;
      comp.seed = lo->seed;
      for (int j = 0; j < std::min<int>(std::max(lo->n_checkpoints, 0), 8); j++) pcts.push_back(lo->checkpoints[j]);
    }
    const bool hybrid = lo && !pcts.empty();
    int rc = learned_trees(v, d_params_bf16, d_ws, ws_bytes, cuda_stream, TNC_LEARNED_CANDIDATES, trees, nullptr,
                           hybrid ? &comp : nullptr, hybrid ? &pcts : nullptr);
    if (rc) return rc;
    tnc_plan_opts fb{};
    if (fallback) fb = *fallback;
    else fb.heuristic = TNC_PLAN_BEST;
    const int cap = fb.rank_cap > 0 ? fb.rank_cap : 32;
    int first_rc = TNC_OK;
    std::string first_msg;
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; i++) {
      // the learned plan, then the heuristic one; the cheaper (max rank, MACs) wins
      auto* pl = new tnc_plan_t();
      pl->net = v[i][0];
      pl->tree = std::move(trees[i]);
      const TreeCost cl = tree_cost(pl->tree);
      if (learned_macs) learned_macs[i] = cl.macs;
      auto* ph = new tnc_plan_t();
      ph->net = v[i][0];
      int rh = plan_tree(ph->net, fb, ph->tree);
      const TreeCost ch = rh == TNC_OK ? tree_cost(ph->tree) : TreeCost{1 << 30, 0, 1e300, 0};
      const bool use_l = cl.max_rank < ch.max_rank || (cl.max_rank == ch.max_rank && cl.macs <= ch.macs);
      tnc_plan_t* keep = use_l ? pl : ph;
      delete (use_l ? ph : pl);
      tnc_plan_stats st{};
      int r = finish_plan(keep, cap, &st);
      if (stats) stats[i] = st;
      if (chose_learned) chose_learned[i] = use_l ? 1 : 0;
      if (r != TNC_OK) {
        delete keep;
        keep = nullptr;
#pragma omp critical
        {
          if (first_rc == TNC_OK) {
            first_rc = r;
            first_msg = "formula " + std::to_string(i) + ": " + tnc_last_error();
          }
        }
      }
      out[i] = keep;
    }
    if (first_rc != TNC_OK) {
      for (int i = 0; i < n; i++) {
        tnc_free_plan(out[i]);
        out[i] = nullptr;
      }
      return set_error(first_rc, first_msg);
    }
    return TNC_OK;
  } catch (const std::bad_alloc&) {
    return set_error(TNC_ERR_NOMEM, "out of host memory");
  }
}

int tnc_plan_learned_many(const tnc_network_t* const* nets, int32_t n, const void* d_params_bf16,
                          const tnc_plan_opts* fallback, void* d_ws, size_t ws_bytes, void* cuda_stream,
                          tnc_plan_t** out, tnc_plan_stats* stats, int32_t* chose_learned, double* learned_macs) {
  clear_error();
  if (!d_params_bf16) return set_error(TNC_ERR_INVALID, "scorer parameters NULL");
  return plan_learned_impl(nets, n, d_params_bf16, nullptr, fallback, d_ws, ws_bytes, cuda_stream, out, stats,
                           chose_learned, learned_macs);
}

int tnc_plan_learned_opts(const tnc_network_t* const* nets, int32_t n, const void* d_params_bf16,
                          const tnc_learned_opts* o, const tnc_plan_opts* fallback, void* d_ws, size_t ws_bytes,
                          void* cuda_stream, tnc_plan_t** out, tnc_plan_stats* stats, int32_t* chose_learned,
                          double* learned_macs) {
  clear_error();
  if (!o) return set_error(TNC_ERR_INVALID, "learned options NULL");
  return plan_learned_impl(nets, n, d_params_bf16, o, fallback, d_ws, ws_bytes, cuda_stream, out, stats,
                           chose_learned, learned_macs);
}

int tnc_learned_dataset_opts(const tnc_network_t* const* nets, int32_t n, const tnc_learned_opts* o,
                             const void* d_params_bf16, void* d_ws, size_t ws_bytes, void* cuda_stream, float* x,
                             float* t, int64_t cap_rows, int64_t* n_rows) {
  clear_error();
  if (!nets || n <= 0 || !o || o->states <= 0 || o->cands <= 1 || !n_rows || (d_params_bf16 && !d_ws))
    return set_error(TNC_ERR_INVALID, "bad dataset arguments");
  try {
    std::vector<const Network*> v;
    for (int i = 0; i < n; i++) {
      if (!nets[i]) return set_error(TNC_ERR_INVALID, "NULL network");
      v.push_back(&nets[i]->net);
    }
    tnc_plan_opts comp{};
    comp.heuristic = o->completion;
    comp.tries = 2;
    comp.seed = o->seed;
    std::vector<std::vector<int>> chosen;
    if (d_params_bf16) {  // follow the learned planner's own merges
      std::vector<Tree> trees;
      int rc = learned_trees(v, d_params_bf16, d_ws, ws_bytes, cuda_stream, TNC_LEARNED_CANDIDATES, trees, &chosen,
                             nullptr, nullptr);
      if (rc) return rc;
    }
    std::vector<float> X, T;
    learned_dataset(v, o->states, o->cands, o->seed, X, T, d_params_bf16 ? &chosen : nullptr,
                    o->completion == TNC_PLAN_GREEDY ? nullptr : &comp, o->max_pct > 0 ? o->max_pct : 100);
    *n_rows = (int64_t)T.size();
    if (!x || !t || cap_rows < (int64_t)T.size())
      return set_error(TNC_ERR_BUFFER, "need " + std::to_string(T.size()) + " rows");
    std::copy(X.begin(), X.end(), x);
    std::copy(T.begin(), T.end(), t);
    return TNC_OK;
  } catch (const std::bad_alloc&) {
    return set_error(TNC_ERR_NOMEM, "out of host memory");
  }
}

}  // extern "C"

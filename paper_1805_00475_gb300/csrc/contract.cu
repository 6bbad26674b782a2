// C ABI, device half.  Contraction of one formula or of a group of formulas
// (tnc_contract, tnc_contract_many, tnc_contract_sliced) runs tree level by
// tree level: one level_kernel launch for the level's small steps of every
// plan of the group, one launch each for its big, one-small-operand and
// split-K steps, and the dense steps on the tensor-core paths (tc.cu,
// tc_p8.cu); then the component product and the CRT.  The allocation-free
// variant (tnc_contract_noalloc) runs the steps in order in a fixed array.
// The persistent batch (tnc_batch_*) contracts many small plans in one
// graph-captured launch of batch_kernel.
#include <type_traits>
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "tnc_internal.h"

using namespace tnc;
using tnc_dev::BatchArgs;
using tnc_dev::CrtConsts;
using tnc_dev::ModGroup;
using tnc_dev::RootMap;

namespace {

#define CUDA_TRY(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return set_error(TNC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

constexpr size_t kAlign = 256;

// An NVTX range for profilers (nvtx is header-only and costs nothing when no
// tool is attached): whole calls, tree levels, dense steps, batch launches.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Dense-step timing of tnc_contract (off unless tnc_set_step_timing(1)).
thread_local bool g_time_dense = false;
thread_local double g_dense_ms = 0.0;
thread_local int g_dense_launches = 0;
thread_local double g_total_ms = 0.0;
thread_local tnc_launch_counts g_launches{};
thread_local std::vector<tnc_dense_step_time> g_dense_steps;  // timing mode: per dense launch
thread_local uint64_t g_h2d_bytes = 0, g_d2h_bytes = 0;  // host <-> device copies of the last contraction
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 148;
  return n;
}

uint32_t powmod(uint64_t a, uint64_t e, uint32_t p) {
  uint64_t r = 1;
  a %= p;
  while (e) {
    if (e & 1) r = r * a % p;
    a = a * a % p;
    e >>= 1;
  }
  return (uint32_t)r;
}

// Residues are processed in groups of 4, 2 or 1 primes (one pass each).
struct Groups {
  std::vector<int> rg, col;
};

Groups split_groups(int R) {
  Groups g;
  int c = 0;
  for (int s : {4, 2, 1})
    while (R - c >= s) {
      g.rg.push_back(s);
      g.col.push_back(c);
      c += s;
    }
  return g;
}

struct Arith {
  int R = 0;
  std::vector<uint32_t> primes;
  CrtConsts crt{};
  double log2_prod = 0;
  Groups groups;
  ModGroup group(int gi) const {
    uint32_t p[4];
    for (int r = 0; r < 4; r++) p[r] = r < groups.rg[gi] ? primes[groups.col[gi] + r] : primes[groups.col[gi]];
    return tnc_dev::make_mod_group(p);
  }
};

int make_arith(const tnc_contract_opts* o, Arith& a) {
  if (!o) return set_error(TNC_ERR_INVALID, "contract opts NULL");
  if (o->path != TNC_PATH_INT64 && o->path != TNC_PATH_TC && o->path != TNC_PATH_TC_P8)
    return set_error(TNC_ERR_INVALID, "unknown arithmetic path");
  const bool p8 = o->path == TNC_PATH_TC_P8;
  const int max_r = p8 ? kP8MaxResidues : 16;
  if (o->n_residues < 1 || o->n_residues > max_r)
    return set_error(TNC_ERR_INVALID, p8 ? "n_residues must be in [1, 53]" : "n_residues must be in [1, 16]");
  a.R = o->n_residues;
  if (o->primes) {
    a.primes.assign(o->primes, o->primes + a.R);
    for (int i = 0; i < a.R; i++) {
      uint32_t p = a.primes[i];
      if (p8 ? (p < 3 || p > kP8PrimeMax || !is_prime_u32(p))
             : (p <= (1u << 29) || p >= (1u << 31) || !is_prime_u32(p)))
        return set_error(TNC_ERR_INVALID, p8 ? "primes must be primes in [3, 251]" : "primes must be primes in (2^29, 2^31)");
      for (int j = 0; j < i; j++)
        if (a.primes[j] == p) return set_error(TNC_ERR_INVALID, "primes must be distinct");
    }
  } else {
    a.primes = p8 ? default_primes_p8(a.R) : default_primes(a.R);
  }
  a.crt = CrtConsts{};
  a.crt.R = a.R;
  a.log2_prod = 0;
  for (int i = 0; i < a.R; i++) {
    const uint32_t p = a.primes[i];
    a.crt.p[i] = p;
    a.crt.mu[i] = ~0ull / p;
    uint64_t prod = 1;
    for (int j = 0; j < i; j++) prod = prod * (a.primes[j] % p) % p;
    a.crt.inv[i] = i == 0 ? 1u : powmod(prod, p - 2, p);
    a.log2_prod += std::log2((double)p);
  }
  // limbs of the CRT value: enough for prod p < 2^(32 n_limbs)
  a.crt.n_limbs = p8 ? (int)std::floor(a.log2_prod / 32.0) + 1 : (31 * a.R + 31) / 32;
  a.groups = split_groups(a.R);
  return TNC_OK;
}

uint32_t result_flags(const tnc_plan_t* p, const Arith& a) {
  return p->net.log2_bound >= a.log2_prod - 1e-9 ? TNC_MAYBE_WRAPPED : 0u;
}

// The word type of a residue in a pass (u32, or a byte on the 8-bit-prime path).
template <typename T>
struct WordTag {
  using type = T;
};

template <typename F>
int dispatch_rg(int rg, F&& f) {
  switch (rg) {
    case 4: return f(std::integral_constant<int, 4>());
    case 2: return f(std::integral_constant<int, 2>());
    default: return f(std::integral_constant<int, 1>());
  }
}

// ---------------------------------------------------------------- single formula

// Workspace of a group of plans contracted together (one plan: the
// single-formula layout).  Descriptors of all plans side by side; every plan's
// tensors in its own part of one arena (arena_base, in entries, a multiple of
// 64 so that every plan's entries start 16-byte aligned); scratch shared by
// the group's steps, which run one after another on one stream.
struct SeqLayout {
  size_t off_leaves, off_tables, off_steps, off_small, off_tc, off_err, off_part, off_results, off_limbs, off_p8,
      off_arena, total;
  uint64_t n_out;  // result entries of the whole group
  size_t n_dense;
  std::vector<uint64_t> arena_base, res_base, leaf_base, table_base;
};

using tnc_dev::GridStep;

// Launch shape of a grid-wide step: S = threads * blocks = 2^s <= 2^c.
void grid_shape(int c, int* threads, int* blocks, int* s) {
  const int t = c >= 8 ? 8 : c;
  const int b = c >= 8 ? std::min(c - 8, 10) : 0;
  *threads = 1 << t;
  *blocks = 1 << b;
  *s = t + b;
}

// Split-K for steps with at most 2^12 outputs and at least 2^9 shared values:
// returns log2 of the number of K slices (0 = no split).  A block sums one
// slice of one output: slices keep at least 256 shared values (one per
// thread), the grid aims at 2^10 blocks (about 7 per SM; a final dot product
// of two rank-22 tensors then sums 16 values per thread instead of one) and
// keeps at least two slices; outputs x slices stays at most 2^13.  (Capping
// the values per thread at 64 with more slices measured 6 % slower on the
// 1-in-3 batch's heavy formulas and no faster on C4-sized ones.)
uint32_t splitk_log(const StepDesc& d) {
  if (d.c > 12 || d.k < 9) return 0;
  const uint32_t ls = d.c < 9 ? 10u - d.c : 1u;
  return std::min<uint32_t>(ls, d.k - 8u);
}

GridStep make_grid_step(const StepDesc& d) {
  GridStep g;
  std::memset(&g, 0, sizeof(g));
  g.d = d;
  int op[64] = {0}, dst[64] = {0};
  if (d.nra != TNC_BITMAP) {
    for (int i = 0; i < d.nra; i++)
      for (int q = 0; q < d.map.runs.ra[i].len; q++) {
        op[d.map.runs.ra[i].src + q] = 0;
        dst[d.map.runs.ra[i].src + q] = d.map.runs.ra[i].dst + q;
      }
    for (int i = 0; i < d.nrb; i++)
      for (int q = 0; q < d.map.runs.rb[i].len; q++) {
        op[d.map.runs.rb[i].src + q] = 1;
        dst[d.map.runs.rb[i].src + q] = d.map.runs.rb[i].dst + q;
      }
  } else {
    for (int j = 0; j < d.c; j++) {
      op[j] = d.map.bit[j] >> 7;
      dst[j] = d.map.bit[j] & 63;
    }
  }
  for (int j = 0; j < d.c; j++) {
    g.wA[j] = op[j] == 0 ? 1ull << dst[j] : 0ull;
    g.wB[j] = op[j] == 1 ? 1ull << dst[j] : 0ull;
  }
  int threads, blocks, sh;
  grid_shape(d.c, &threads, &blocks, &sh);
  g.s = (uint32_t)sh;
  for (int t = sh; t < d.c; t++) {
    uint64_t sa = 0, sb = 0;
    for (int j = sh; j < t; j++) {
      sa += g.wA[j];
      sb += g.wB[j];
    }
    g.dA[t] = g.wA[t] - sa;
    g.dB[t] = g.wB[t] - sb;
  }
  return g;
}

// A big step with one small operand (at most 2^4 free rows, at most 2^3
// shared values) runs as outer_kernel: the small operand staged in shared
// memory, one row of the large operand per thread.
bool outer_eligible(const StepDesc& d) {
  return splitk_log(d) == 0 && d.c >= 16 && std::min(d.ka, d.kb) <= 4 && std::max(d.ka, d.kb) <= 32 && d.k <= 3;
}

tnc_dev::OuterStep make_outer_step(const StepDesc& d) {
  tnc_dev::OuterStep o;
  std::memset(&o, 0, sizeof(o));
  const int s_side = d.ka <= d.kb ? 0 : 1;  // the small operand: A, or B
  o.fs = s_side ? d.kb : d.ka;
  o.fl = s_side ? d.ka : d.kb;
  o.k = d.k;
  o.s_off = s_side ? d.b_off : d.a_off;
  o.l_off = s_side ? d.a_off : d.b_off;
  o.c_off = d.c_off;
  int op[64] = {0}, dst[64] = {0};
  if (d.nra != TNC_BITMAP) {
    for (int i = 0; i < d.nra; i++)
      for (int q = 0; q < d.map.runs.ra[i].len; q++) {
        op[d.map.runs.ra[i].src + q] = 0;
        dst[d.map.runs.ra[i].src + q] = d.map.runs.ra[i].dst + q;
      }
    for (int i = 0; i < d.nrb; i++)
      for (int q = 0; q < d.map.runs.rb[i].len; q++) {
        op[d.map.runs.rb[i].src + q] = 1;
        dst[d.map.runs.rb[i].src + q] = d.map.runs.rb[i].dst + q;
      }
  } else {
    for (int j = 0; j < d.c; j++) {
      op[j] = d.map.bit[j] >> 7;
      dst[j] = d.map.bit[j] & 63;
    }
  }
  uint64_t wS[4] = {0, 0, 0, 0};
  for (int j = 0; j < d.c; j++) {
    if (op[j] == s_side) wS[dst[j]] = 1ull << j;
    else o.oL[dst[j]] = 1ull << j;
  }
  for (uint32_t x = 0; x < (1u << o.fs); x++)
    for (uint32_t i = 0; i < o.fs; i++)
      if ((x >> i) & 1u) o.oS[x] += wS[i];
  o.contig = 1;
  for (uint32_t i = 0; i < o.fs; i++)
    if (wS[i] != (1ull << i)) o.contig = 0;
  return o;
}

// What one plan adds to a group's workspace: counts of descriptors, result
// entries and arena entries (summed over the group), and scratch bytes (the
// group's maximum).
struct Foot {
  size_t leaves = 0, tables = 0, nseq = 0, nlvl = 0, n_dense = 0;
  uint64_t n_out = 0, arena = 0, part = 0, p8 = 0;
  void add(const Foot& f) {
    leaves += f.leaves;
    tables += f.tables;
    nseq += f.nseq;
    nlvl += f.nlvl;
    n_dense += f.n_dense;
    n_out += f.n_out;
    arena += f.arena;
    part = std::max(part, f.part);
    p8 = std::max(p8, f.p8);
  }
};

Foot foot_of(const tnc_plan_t* p, int R, int path) {
  const int rg_max = R >= 4 ? 4 : (R >= 2 ? 2 : 1);
  Foot f;
  f.leaves = p->low.leaves.size();
  f.tables = p->low.leaf_tables.size();
  f.nseq = p->low.seq_steps.size();
  f.nlvl = p->low.lvl_steps.size();
  f.n_out = 1ull << p->net.open_vars.size();
  for (const StepDesc& d : p->low.seq_steps) f.n_dense += tc_eligible(d) ? 1 : 0;
  for (const StepDesc& d : p->low.lvl_steps) {
    if (splitk_log(d) > 0)
      f.part = std::max<uint64_t>(f.part, (1ull << (d.c + splitk_log(d))) * rg_max * sizeof(uint32_t));
    if (tc_eligible(d) && tc_split_log(d) > 0)
      f.part = std::max<uint64_t>(f.part, (1ull << (d.c + tc_split_log(d))) * sizeof(uint32_t));
    if (path == TNC_PATH_TC_P8 && p8_eligible(d)) {
      f.part = std::max<uint64_t>(f.part, p8_part_bytes(d, rg_max));
      f.p8 = std::max<uint64_t>(f.p8, p8_scratch_bytes(d, rg_max));
    }
  }
  uint64_t arena = std::max(p->low.seq_arena_entries, p->low.lvl_arena_entries);
  if (path == TNC_PATH_TC_P8) arena = std::max(arena, p->low.p8_arena_entries);
  f.arena = (arena + 63) / 64 * 64;
  return f;
}

// Offsets of the workspace sections for the group footprint f.
SeqLayout layout_of(const Foot& f, int R, int path) {
  SeqLayout s{};
  const int rg_max = R >= 4 ? 4 : (R >= 2 ? 2 : 1);
  size_t o = 0;
  auto sect = [&](size_t& off, size_t bytes) {
    off = o;
    o = align_up(o + bytes);
  };
  sect(s.off_leaves, f.leaves * sizeof(LeafDesc));
  sect(s.off_tables, f.tables * sizeof(uint32_t));
  sect(s.off_steps, std::max(f.nseq, f.nlvl) * sizeof(GridStep));
  sect(s.off_small, f.nlvl * sizeof(StepDesc));
  sect(s.off_tc, f.n_dense * R * tc_step_bytes());
  sect(s.off_err, 64);
  sect(s.off_part, f.part);
  sect(s.off_results, f.n_out * R * sizeof(uint32_t));
  sect(s.off_limbs, f.n_out * ((31 * R + 31) / 32) * sizeof(uint32_t));
  sect(s.off_p8, f.p8);
  const size_t word = path == TNC_PATH_TC_P8 ? 1 : sizeof(uint32_t);  // bytes per residue
  sect(s.off_arena, f.arena * rg_max * word);
  s.total = o;
  s.n_out = f.n_out;
  s.n_dense = f.n_dense;
  return s;
}

SeqLayout group_layout(const tnc_plan_t* const* plans, int n, int R, int path = TNC_PATH_INT64) {
  Foot sum;
  std::vector<uint64_t> arena_base, res_base, leaf_base, table_base;
  for (int i = 0; i < n; i++) {
    const Foot f = foot_of(plans[i], R, path);
    leaf_base.push_back(sum.leaves);
    table_base.push_back(sum.tables);
    res_base.push_back(sum.n_out);
    arena_base.push_back(sum.arena);
    sum.add(f);
  }
  SeqLayout s = layout_of(sum, R, path);
  s.arena_base = std::move(arena_base);
  s.res_base = std::move(res_base);
  s.leaf_base = std::move(leaf_base);
  s.table_base = std::move(table_base);
  return s;
}

// Consecutive groups of the plans whose workspace each fits `budget` bytes
// (every plan alone must fit): [begin, end) ranges.
int plan_groups(const tnc_plan_t* const* plans, int n, int R, int path, size_t budget,
                std::vector<std::pair<int, int>>& out) {
  out.clear();
  int b = 0;
  Foot sum;
  for (int i = 0; i < n; i++) {
    Foot f = foot_of(plans[i], R, path);
    Foot t = sum;
    t.add(f);
    if (i > b && layout_of(t, R, path).total > budget) {
      out.push_back({b, i});
      b = i;
      sum = Foot();
      t = f;
    }
    if (layout_of(t, R, path).total > budget)
      return set_error(TNC_ERR_BUFFER, "plan " + std::to_string(i) + " alone needs " +
                                           std::to_string(layout_of(t, R, path).total) + " bytes of workspace");
    sum = t;
  }
  if (b < n) out.push_back({b, n});
  return TNC_OK;
}

SeqLayout seq_layout(const tnc_plan_t* p, int R, int path = TNC_PATH_INT64) { return group_layout(&p, 1, R, path); }

int fill_count(tnc_count* out, uint64_t n_out, const Arith& a, const uint32_t* res, const uint32_t* limbs,
               uint32_t flags) {
  out->n_out = (int32_t)n_out;
  out->n_limbs = a.crt.n_limbs;
  out->flags = flags;
  if (out->cap_out < (int32_t)n_out) return set_error(TNC_ERR_BUFFER, "count buffer holds fewer entries than 2^n_open");
  if (out->residues) std::memcpy(out->residues, res, n_out * a.R * sizeof(uint32_t));
  if (out->limbs) {
    if (out->cap_limbs < a.crt.n_limbs) return set_error(TNC_ERR_BUFFER, "need " + std::to_string(a.crt.n_limbs) + " limbs");
    for (uint64_t e = 0; e < n_out; e++) {
      std::memset(out->limbs + e * out->cap_limbs, 0, out->cap_limbs * sizeof(uint32_t));
      std::memcpy(out->limbs + e * out->cap_limbs, limbs + e * a.crt.n_limbs, a.crt.n_limbs * sizeof(uint32_t));
    }
  }
  return TNC_OK;
}

}  // namespace

extern "C" size_t tnc_workspace_bytes(const tnc_plan_t* plan, int32_t n_residues) {
  if (!plan || n_residues < 1 || n_residues > 16) return 0;
  return seq_layout(plan, n_residues).total;
}

extern "C" void tnc_set_step_timing(int32_t on) { g_time_dense = on != 0; }

extern "C" int tnc_last_dense_time(double* ms, int32_t* n_steps) {
  if (ms) *ms = g_dense_ms;
  if (n_steps) *n_steps = g_dense_launches;
  return TNC_OK;
}

extern "C" int tnc_last_dense_steps(tnc_dense_step_time* out, int32_t cap, int32_t* n) {
  if (n) *n = (int32_t)g_dense_steps.size();
  if (!out) return TNC_OK;
  if (cap < (int32_t)g_dense_steps.size())
    return set_error(TNC_ERR_BUFFER, "need " + std::to_string(g_dense_steps.size()) + " entries");
  std::copy(g_dense_steps.begin(), g_dense_steps.end(), out);
  return TNC_OK;
}

extern "C" int tnc_last_contract_time(double* device_ms) {
  if (device_ms) *device_ms = g_total_ms;
  return TNC_OK;
}

tnc_launch_counts& tnc::launch_counts() { return g_launches; }

extern "C" int tnc_last_launch_counts(tnc_launch_counts* out) {
  if (!out) return set_error(TNC_ERR_INVALID, "NULL argument");
  *out = g_launches;
  return TNC_OK;
}

extern "C" int tnc_last_io_bytes(uint64_t* h2d_bytes, uint64_t* d2h_bytes) {
  if (h2d_bytes) *h2d_bytes = g_h2d_bytes;
  if (d2h_bytes) *d2h_bytes = g_d2h_bytes;
  return TNC_OK;
}

extern "C" size_t tnc_workspace_bytes_opts(const tnc_plan_t* plan, const tnc_contract_opts* opts) {
  clear_error();
  Arith a;
  if (!plan || make_arith(opts, a)) return 0;
  return seq_layout(plan, a.R, opts->path).total;
}

// Residues r of a sum of contractions: acc[e R + r] = (acc + src) mod p_r.
__global__ void residue_add_kernel(uint32_t* __restrict__ acc, const uint32_t* __restrict__ src, uint64_t n, int R,
                                   CrtConsts cc) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t p = cc.p[i % R];
    const uint32_t s = acc[i] + src[i];  // both below p < 2^31
    acc[i] = s >= p ? s - p : s;
  }
}

// The contraction of a group of plans, their tree levels merged: level l of
// every plan of the group runs together (one launch for all their steps with
// fewer than 2^16 outputs, one launch each for big, split-K and dense steps).
// With sum_into == nullptr every plan's count is finished (CRT, copy to
// outs[i]); otherwise the residues [2^n_open][R] of every plan are added into
// the device buffer sum_into (the plans are the slices of one count) and
// nothing else is returned.
static int contract_group(const tnc_plan_t* const* plans, int n, const tnc_contract_opts* opts, void* dev_ws,
                          size_t ws_bytes, void* cuda_stream, tnc_count* outs, uint32_t* sum_into) {
  if (!plans || n <= 0 || (!outs && !sum_into)) return set_error(TNC_ERR_INVALID, "NULL argument");
  for (int i = 0; i < n; i++)
    if (!plans[i]) return set_error(TNC_ERR_INVALID, "NULL plan");
  Arith a;
  int rc = make_arith(opts, a);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // empty networks (the empty product, 1) are answered on the host
  std::vector<const tnc_plan_t*> work;
  std::vector<int> work_idx;
  for (int i = 0; i < n; i++) {
    if (!plans[i]->tree.nodes.empty()) {
      work.push_back(plans[i]);
      work_idx.push_back(i);
      continue;
    }
    std::vector<uint32_t> res(a.R, 1u), limbs(a.crt.n_limbs, 0u);
    limbs[0] = 1;
    if (sum_into) {
      if (!dev_ws || ws_bytes < (size_t)a.R * 4) return set_error(TNC_ERR_BUFFER, "workspace too small");
      CUDA_TRY(cudaMemcpyAsync(dev_ws, res.data(), a.R * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
      residue_add_kernel<<<1, 64, 0, st>>>(sum_into, (const uint32_t*)dev_ws, (uint64_t)a.R, a.R, a.crt);
      CUDA_TRY(cudaGetLastError());
      CUDA_TRY(cudaStreamSynchronize(st));
    } else {
      rc = fill_count(&outs[i], 1, a, res.data(), limbs.data(), 0);
      if (rc) return rc;
    }
  }
  if (work.empty()) return TNC_OK;
  const int nw = (int)work.size();
  const SeqLayout L = group_layout(work.data(), nw, a.R, opts->path);
  if (!dev_ws || ws_bytes < L.total) return set_error(TNC_ERR_BUFFER, "workspace smaller than tnc_workspace_bytes");
  if (((uintptr_t)dev_ws) % kAlign) return set_error(TNC_ERR_INVALID, "workspace must be 256-byte aligned");
  if (inject_hit(TNC_INJECT_LAUNCH)) return set_error(TNC_ERR_CUDA, "injected failure (TNC_INJECT_LAUNCH)");
  char* ws = (char*)dev_ws;
  // Every plan runs level by level (the tree-level schedule of the lowering);
  // offsets are shifted to the plan's part of the group's arena, tables and
  // results.
  const bool p8 = opts->path == TNC_PATH_TC_P8;
  const bool tc = opts->path == TNC_PATH_TC || p8;
  std::vector<LeafDesc> leaves;
  std::vector<uint32_t> tables;
  size_t n_lev = 0;
  for (int w = 0; w < nw; w++) {
    const Lowered& lw = work[w]->low;
    for (size_t i = 0; i < lw.leaves.size(); i++) {
      LeafDesc ld = lw.leaves[i];
      ld.off = (p8 ? lw.p8_leaf_off[i] : lw.lvl_leaf_off[i]) + L.arena_base[w];
      ld.table_off += (uint32_t)L.table_base[w];
      leaves.push_back(ld);
    }
    tables.insert(tables.end(), lw.leaf_tables.begin(), lw.leaf_tables.end());
    n_lev = std::max(n_lev, lw.lvl_start.empty() ? (size_t)0 : lw.lvl_start.size() - 1);
  }
  CUDA_TRY(cudaMemcpyAsync(ws + L.off_leaves, leaves.data(), leaves.size() * sizeof(LeafDesc), cudaMemcpyHostToDevice, st));
  if (!tables.empty())
    CUDA_TRY(cudaMemcpyAsync(ws + L.off_tables, tables.data(), tables.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                             st));
  g_h2d_bytes += leaves.size() * sizeof(LeafDesc) + tables.size() * sizeof(uint32_t);
  // the group's steps by level: small ones (one index space per level across
  // the plans), big, split-K and dense ones (one launch each)
  enum Kind { kGrid, kSplit, kTc, kOuter };
  struct Big {
    int kind, slot;
    StepDesc d;      // offsets shifted to the group's arena
    uint32_t flags;  // p8: direct fp16 planes (kP8Direct*)
  };
  std::vector<std::vector<Big>> big(n_lev);
  std::vector<GridStep> gsteps;
  std::vector<tnc_dev::OuterStep> outers;
  std::vector<StepDesc> small;
  std::vector<uint32_t> small_lo(n_lev), small_hi(n_lev), small_work(n_lev);
  std::vector<char> tcbuf;
  size_t nd = 0;
  for (size_t l = 0; l < n_lev; l++) {
    small_lo[l] = (uint32_t)small.size();
    uint64_t wk = 0;
    for (int w = 0; w < nw; w++) {
      const Lowered& lw = work[w]->low;
      if (l + 1 >= lw.lvl_start.size()) continue;
      const uint64_t base = L.arena_base[w];
      for (uint32_t i = lw.lvl_start[l]; i < lw.lvl_start[l + 1]; i++) {
        StepDesc d = p8 ? lw.p8_steps[i] : lw.lvl_steps[i];
        d.a_off += base;
        d.b_off += base;
        d.c_off += base;
        uint32_t flags = 0;
        if (p8) {
          const int sa = lw.lvl_src_a[i], sb = lw.lvl_src_b[i];
          if (lw.p8_direct[i]) flags |= kP8DirectOut;
          if (sa >= 0 && lw.p8_direct[sa]) flags |= kP8DirectA;
          if (sb >= 0 && lw.p8_direct[sb]) flags |= kP8DirectB;
        }
        if (tc && (p8 ? p8_eligible(d) : tc_eligible(d))) {
          big[l].push_back(Big{kTc, (int)nd++, d, flags});
        } else if (flags) {
          return set_error(TNC_ERR_INVALID, "internal: direct fp16 planes on a CUDA-core step");
        } else if (outer_eligible(d)) {
          big[l].push_back(Big{kOuter, (int)outers.size(), d, 0});
          outers.push_back(make_outer_step(d));
        } else if (splitk_log(d) > 0 || d.c >= 16) {
          big[l].push_back(Big{splitk_log(d) > 0 ? kSplit : kGrid, (int)gsteps.size(), d, 0});
          gsteps.push_back(make_grid_step(d));
        } else {
          d.work_lo = (uint32_t)wk;
          wk += 1u << d.c;
          small.push_back(d);
        }
      }
    }
    if (wk >= (1ull << 32)) return set_error(TNC_ERR_TOO_LARGE, "a merged level has more than 2^32 small outputs");
    small_hi[l] = (uint32_t)small.size();
    small_work[l] = (uint32_t)wk;
  }
  g_h2d_bytes += gsteps.size() * sizeof(GridStep) + small.size() * sizeof(StepDesc);
  if (!gsteps.empty())
    CUDA_TRY(cudaMemcpyAsync(ws + L.off_steps, gsteps.data(), gsteps.size() * sizeof(GridStep), cudaMemcpyHostToDevice,
                             st));
  if (!small.empty())
    CUDA_TRY(cudaMemcpyAsync(ws + L.off_small, small.data(), small.size() * sizeof(StepDesc), cudaMemcpyHostToDevice, st));
  if (nd && !p8) {
    tcbuf.assign(nd * a.R * tc_step_bytes(), 0);
    for (size_t l = 0; l < n_lev; l++)
      for (const Big& b : big[l])
        if (b.kind == kTc)
          for (int r = 0; r < a.R; r++)
            tc_make_step(b.d, a.primes[r], tcbuf.data() + ((size_t)b.slot * a.R + r) * tc_step_bytes());
    CUDA_TRY(cudaMemcpyAsync(ws + L.off_tc, tcbuf.data(), tcbuf.size(), cudaMemcpyHostToDevice, st));
    g_h2d_bytes += tcbuf.size();
  }
  // residue groups: limb tensor-core passes carry one residue per entry; the
  // 8-bit-prime path keeps groups of 4 and runs its dense steps per residue
  Groups groups = a.groups;
  if (tc && !p8) {
    groups = Groups();
    for (int r = 0; r < a.R; r++) {
      groups.rg.push_back(1);
      groups.col.push_back(r);
    }
  }
  uint32_t* d_err = (uint32_t*)(ws + L.off_err);
  CUDA_TRY(cudaMemsetAsync(d_err, 0, 64, st));
  // dense-step events (tnc_set_step_timing), destroyed on every return
  std::vector<cudaEvent_t> dense_events;
  std::vector<tnc_dense_step_time> dense_info;  // shapes of the timed dense launches
  struct EventGuard {
    std::vector<cudaEvent_t>& v;
    ~EventGuard() {
      for (cudaEvent_t e : v) cudaEventDestroy(e);
    }
  } event_guard{dense_events};
  cudaEvent_t whole[2] = {nullptr, nullptr};  // the device work of the whole contraction (timing mode)
  if (g_time_dense) {
    CUDA_TRY(cudaEventCreate(&whole[0]));
    CUDA_TRY(cudaEventCreate(&whole[1]));
    dense_events.push_back(whole[0]);
    dense_events.push_back(whole[1]);
    CUDA_TRY(cudaEventRecord(whole[0], st));
  }
  const GridStep* d_steps = (const GridStep*)(ws + L.off_steps);
  const StepDesc* d_small = (const StepDesc*)(ws + L.off_small);
  uint32_t* results = (uint32_t*)(ws + L.off_results);
  uint32_t* part = (uint32_t*)(ws + L.off_part);
  std::vector<RootMap> rms(nw);
  std::vector<uint64_t> root_off(nw);
  for (int w = 0; w < nw; w++) {
    const Lowered& lw = work[w]->low;
    rms[w] = RootMap{};
    rms[w].n_open = (int)work[w]->net.open_vars.size();
    for (int j = 0; j < rms[w].n_open; j++) rms[w].perm[j] = lw.root_perm[j];
    root_off[w] = L.arena_base[w] + (lw.lvl_steps.empty() ? (p8 ? lw.p8_leaf_off : lw.lvl_leaf_off)[work[w]->tree.root]
                                                          : (p8 ? lw.p8_root_off : lw.lvl_root_off));
  }
  const int sms = sm_count();
  for (size_t gi = 0; gi < groups.rg.size(); gi++) {
    uint32_t gp[4];
    for (int r = 0; r < 4; r++) gp[r] = r < groups.rg[gi] ? a.primes[groups.col[gi] + r] : a.primes[groups.col[gi]];
    const ModGroup mg = tnc_dev::make_mod_group(gp);
    // one pass over the residue group; the 8-bit-prime path stores a residue
    // per byte
    auto pass = [&](auto rgc, auto wtag, auto n30tag) -> int {
      constexpr int RG = decltype(rgc)::value;
      using W = typename decltype(wtag)::type;
      constexpr bool N30 = decltype(n30tag)::value;
      W* arena = reinterpret_cast<W*>(ws + L.off_arena);
      const int nl = (int)leaves.size();
      tnc_dev::leaf_fill_kernel<RG, W><<<std::min(nl, sms * 8), 64, 0, st>>>(
          (const LeafDesc*)(ws + L.off_leaves), nl, (const uint32_t*)(ws + L.off_tables), arena, mg);
      g_launches.leaf_fill++;
      for (size_t l = 0; l < n_lev; l++) {
        NvtxRange level_range("tnc level");
        const uint32_t n_small = small_hi[l] - small_lo[l];
        if (n_small) {
          const uint32_t wk = small_work[l];
          const unsigned blocks = (unsigned)std::min<uint64_t>((wk + 255) / 256, (uint64_t)sms * 8);
          tnc_dev::level_kernel<RG, W, N30><<<blocks, 256, 0, st>>>(d_small + small_lo[l], n_small, wk, arena, mg);
          g_launches.level++;
        }
        for (const Big& b : big[l]) {
          if (b.kind == kTc) {
            NvtxRange dense_range("tnc dense step");
            if (RG != 1 && !p8) return set_error(TNC_ERR_INVALID, "internal: tensor-core step in a multi-residue pass");
            int rc2 = TNC_OK;
            cudaEvent_t ev[2] = {nullptr, nullptr};
            if (g_time_dense) {
              CUDA_TRY(cudaEventCreate(&ev[0]));
              CUDA_TRY(cudaEventCreate(&ev[1]));
              CUDA_TRY(cudaEventRecord(ev[0], st));
            }
            if (p8) {
              rc2 = p8_launch(b.d, a.primes.data() + groups.col[gi], RG, reinterpret_cast<uint8_t*>(arena),
                              (uint64_t)(L.total - L.off_arena), b.flags, ws + L.off_p8,
                              reinterpret_cast<uint8_t*>(part), d_err, sms, st);
            } else {
              const char* dstep = ws + L.off_tc + ((size_t)b.slot * a.R + groups.col[gi]) * tc_step_bytes();
              rc2 = tc_launch(dstep, b.d, reinterpret_cast<uint32_t*>(arena), part, d_err, st);
            }
            if (g_time_dense) {
              CUDA_TRY(cudaEventRecord(ev[1], st));
              dense_events.push_back(ev[0]);
              dense_events.push_back(ev[1]);
              tnc_dense_step_time info{};
              info.macs = std::ldexp(1.0, b.d.ka + b.d.kb + b.d.k);
              info.rows_log2 = b.d.ka;
              info.cols_log2 = b.d.kb;
              info.k_log2 = b.d.k;
              info.residues = RG;
              info.tile_n = p8 ? (int32_t)p8_tile_width(b.d) : 32;
              info.log_split = (int32_t)(p8 ? p8_split_log(b.d) : tc_split_log(b.d));
              dense_info.push_back(info);
            }
            if (rc2) return rc2;
          } else if (b.kind == kOuter) {
            const tnc_dev::OuterStep& os = outers[b.slot];
            const unsigned blocks = (unsigned)std::min<uint64_t>(((1ull << os.fl) + 255) / 256, (uint64_t)sms * 8);
            tnc_dev::outer_kernel<RG, W, N30><<<blocks, 256, 0, st>>>(os, arena, mg);
            g_launches.outer++;
          } else if (b.kind == kSplit) {
            const uint32_t ls = splitk_log(b.d);
            const uint64_t nblk = 1ull << (b.d.c + ls);
            tnc_dev::splitk_partial_kernel<RG, W, N30><<<(unsigned)nblk, 256, 0, st>>>(d_steps + b.slot, arena, part, ls,
                                                                                       mg);
            tnc_dev::splitk_final_kernel<RG, W, N30><<<(unsigned)(1ull << b.d.c), 256, 0, st>>>(d_steps + b.slot, arena,
                                                                                              part, ls, mg);
            g_launches.splitk++;
          } else {
            int threads, blocks, sh;
            grid_shape(b.d.c, &threads, &blocks, &sh);
            tnc_dev::step_kernel<RG, W, N30><<<blocks, threads, 0, st>>>(d_steps + b.slot, arena, mg);
            g_launches.grid_step++;
          }
        }
      }
      for (int w = 0; w < nw; w++) {
        const uint64_t no = 1ull << rms[w].n_open;
        tnc_dev::extract_kernel<RG, W><<<(unsigned)std::min<uint64_t>((no + 255) / 256, 1024), 256, 0, st>>>(
            arena, root_off[w], rms[w], results + L.res_base[w] * a.R, a.R, groups.col[gi]);
        g_launches.extract++;
      }
      CUDA_TRY(cudaGetLastError());
      return TNC_OK;
    };
    rc = dispatch_rg(groups.rg[gi], [&](auto rgc) -> int {
      if (p8) return pass(rgc, WordTag<uint8_t>(), std::false_type());
      return mg.near30 ? pass(rgc, WordTag<uint32_t>(), std::true_type())
                       : pass(rgc, WordTag<uint32_t>(), std::false_type());
    });
    if (rc) return rc;
  }
  uint32_t h_err = 0;
  if (sum_into) {  // terms of a sum: add every plan's residues, check the device status
    for (int w = 0; w < nw; w++) {
      const uint64_t m = (1ull << rms[w].n_open) * (uint64_t)a.R;
      residue_add_kernel<<<(unsigned)std::min<uint64_t>((m + 255) / 256, 1024), 256, 0, st>>>(
          sum_into, results + L.res_base[w] * a.R, m, a.R, a.crt);
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    g_d2h_bytes += sizeof(uint32_t);
    CUDA_TRY(cudaStreamSynchronize(st));
    if (inject_hit(TNC_INJECT_TIMEOUT)) h_err = 1;
    if (h_err) return set_error(TNC_ERR_TIMEOUT, "a tensor-core step timed out waiting for its MMAs");
    return TNC_OK;
  }
  uint32_t* limbs = (uint32_t*)(ws + L.off_limbs);
  tnc_dev::crt_kernel<<<(unsigned)std::min<uint64_t>((L.n_out + 127) / 128, 1024), 128, 0, st>>>(results, L.n_out, a.crt,
                                                                                                  limbs);
  g_launches.crt++;
  CUDA_TRY(cudaGetLastError());
  if (g_time_dense) CUDA_TRY(cudaEventRecord(whole[1], st));
  CUDA_TRY(cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  std::vector<uint32_t> h_res(L.n_out * a.R), h_limbs(L.n_out * a.crt.n_limbs);
  CUDA_TRY(cudaMemcpyAsync(h_res.data(), results, h_res.size() * 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(h_limbs.data(), limbs, h_limbs.size() * 4, cudaMemcpyDeviceToHost, st));
  g_d2h_bytes += sizeof(uint32_t) + (h_res.size() + h_limbs.size()) * 4;
  CUDA_TRY(cudaStreamSynchronize(st));
  if (inject_hit(TNC_INJECT_TIMEOUT)) h_err = 1;
  if (h_err) return set_error(TNC_ERR_TIMEOUT, "a tensor-core step timed out waiting for its MMAs");
  for (size_t e = 0; e + 1 < dense_events.size(); e += 2) {  // pair 0: the whole contraction
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, dense_events[e], dense_events[e + 1]));
    if (e == 0) {
      g_total_ms += ms;
      continue;
    }
    g_dense_ms += ms;
    g_dense_launches++;
    tnc_dense_step_time info = dense_info[e / 2 - 1];
    info.ms = ms;
    g_dense_steps.push_back(info);
  }
  for (int w = 0; w < nw; w++) {
    rc = fill_count(&outs[work_idx[w]], 1ull << rms[w].n_open, a, h_res.data() + L.res_base[w] * a.R,
                    h_limbs.data() + L.res_base[w] * a.crt.n_limbs, result_flags(work[w], a));
    if (rc) return rc;
  }
  return TNC_OK;
}

// Resets the per-call records (launch counts, copies, timing) of the calling
// thread.
static void reset_records() {
  g_launches = tnc_launch_counts{};
  g_h2d_bytes = g_d2h_bytes = 0;
  g_dense_ms = 0.0;
  g_dense_launches = 0;
  g_total_ms = 0.0;
  g_dense_steps.clear();
}

extern "C" int tnc_contract(const tnc_plan_t* plan, const tnc_contract_opts* opts, void* dev_ws, size_t ws_bytes,
                            void* cuda_stream, tnc_count* out) {
  clear_error();
  reset_records();
  NvtxRange range("tnc_contract");
  if (!plan || !out) return set_error(TNC_ERR_INVALID, "NULL argument");
  return contract_group(&plan, 1, opts, dev_ws, ws_bytes, cuda_stream, out, nullptr);
}

// Slices of one count: the sum of the plans' counts (each plan the network of
// the formula with some variables fixed), exact as residues, one CRT at the end.
static size_t sliced_head_bytes(uint64_t n_out, const Arith& a) {
  return align_up(n_out * a.R * sizeof(uint32_t)) + align_up(n_out * a.crt.n_limbs * sizeof(uint32_t));
}

extern "C" size_t tnc_workspace_bytes_sliced(const tnc_plan_t* const* plans, int32_t n, const tnc_contract_opts* opts) {
  clear_error();
  Arith a;
  if (!plans || n <= 0 || make_arith(opts, a)) return 0;
  size_t body = 256;
  for (int i = 0; i < n; i++) {
    if (!plans[i]) return 0;
    body = std::max(body, seq_layout(plans[i], a.R, opts->path).total);
  }
  return sliced_head_bytes(1ull << plans[0]->net.open_vars.size(), a) + body;
}

extern "C" int tnc_contract_sliced(const tnc_plan_t* const* plans, int32_t n, const tnc_contract_opts* opts,
                                   void* dev_ws, size_t ws_bytes, void* cuda_stream, tnc_count* out) {
  clear_error();
  reset_records();
  NvtxRange range("tnc_contract_sliced");
  if (!plans || n <= 0 || !out || !opts) return set_error(TNC_ERR_INVALID, "NULL argument");
  Arith a;
  int rc = make_arith(opts, a);
  if (rc) return rc;
  const size_t n_open = plans[0] ? plans[0]->net.open_vars.size() : 0;
  double bound = 0;  // log2 of the sum of the slices' certified bounds
  for (int i = 0; i < n; i++) {
    if (!plans[i]) return set_error(TNC_ERR_INVALID, "NULL plan");
    if (plans[i]->net.open_vars.size() != n_open) return set_error(TNC_ERR_INVALID, "slices differ in open variables");
    const double b = plans[i]->net.log2_bound;
    bound = i == 0 ? b : std::max(bound, b) + std::log2(1.0 + std::exp2(-std::fabs(bound - b)));
  }
  const size_t need = tnc_workspace_bytes_sliced(plans, n, opts);
  if (!dev_ws || ws_bytes < need) return set_error(TNC_ERR_BUFFER, "workspace smaller than tnc_workspace_bytes_sliced");
  if (((uintptr_t)dev_ws) % kAlign) return set_error(TNC_ERR_INVALID, "workspace must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const uint64_t n_out = 1ull << n_open;
  char* ws = (char*)dev_ws;
  uint32_t* acc = (uint32_t*)ws;
  uint32_t* limbs = (uint32_t*)(ws + align_up(n_out * a.R * sizeof(uint32_t)));
  const size_t head = sliced_head_bytes(n_out, a);
  CUDA_TRY(cudaMemsetAsync(acc, 0, n_out * a.R * sizeof(uint32_t), st));
  // as many slices at a time as the workspace holds, their levels merged
  std::vector<std::pair<int, int>> grp;
  rc = plan_groups(plans, n, a.R, opts->path, ws_bytes - head, grp);
  if (rc) return rc;
  for (const auto& g : grp) {
    rc = contract_group(plans + g.first, g.second - g.first, opts, ws + head, ws_bytes - head, cuda_stream, nullptr,
                        acc);
    if (rc) return rc;
  }
  tnc_dev::crt_kernel<<<(unsigned)std::min<uint64_t>((n_out + 127) / 128, 1024), 128, 0, st>>>(acc, n_out, a.crt, limbs);
  g_launches.crt++;
  CUDA_TRY(cudaGetLastError());
  std::vector<uint32_t> h_res(n_out * a.R), h_limbs(n_out * a.crt.n_limbs);
  CUDA_TRY(cudaMemcpyAsync(h_res.data(), acc, h_res.size() * 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(h_limbs.data(), limbs, h_limbs.size() * 4, cudaMemcpyDeviceToHost, st));
  g_d2h_bytes += (h_res.size() + h_limbs.size()) * 4;
  CUDA_TRY(cudaStreamSynchronize(st));
  return fill_count(out, n_out, a, h_res.data(), h_limbs.data(), bound >= a.log2_prod - 1e-9 ? TNC_MAYBE_WRAPPED : 0u);
}

extern "C" size_t tnc_workspace_bytes_many(const tnc_plan_t* const* plans, int32_t n, const tnc_contract_opts* opts,
                                           int32_t group) {
  clear_error();
  Arith a;
  if (!plans || n <= 0 || group <= 0 || make_arith(opts, a)) return 0;
  size_t need = 256;
  for (int i = 0; i < n; i += group) {
    const int m = std::min<int>(group, n - i);
    for (int j = i; j < i + m; j++)
      if (!plans[j]) return 0;
    need = std::max(need, group_layout(plans + i, m, a.R, opts->path).total);
  }
  return need;
}

extern "C" int tnc_contract_many(const tnc_plan_t* const* plans, int32_t n, const tnc_contract_opts* opts,
                                 void* dev_ws, size_t ws_bytes, void* cuda_stream, tnc_count* outs) {
  clear_error();
  reset_records();
  NvtxRange range("tnc_contract_many");
  if (!plans || n <= 0 || !outs || !opts) return set_error(TNC_ERR_INVALID, "NULL argument");
  Arith a;
  int rc = make_arith(opts, a);
  if (rc) return rc;
  for (int i = 0; i < n; i++)
    if (!plans[i]) return set_error(TNC_ERR_INVALID, "NULL plan");
  std::vector<std::pair<int, int>> grp;
  rc = plan_groups(plans, n, a.R, opts->path, ws_bytes, grp);
  if (rc) return rc;
  for (const auto& g : grp) {
    rc = contract_group(plans + g.first, g.second - g.first, opts, dev_ws, ws_bytes, cuda_stream, outs + g.first,
                        nullptr);
    if (rc) return rc;
  }
  return TNC_OK;
}

// ======================================================================= batch

using tnc_dev::BForm;
using tnc_dev::BLeaf;
using tnc_dev::BStep;
using tnc_dev::Seg;

struct tnc_batch_s {
  std::vector<const tnc_plan_t*> plans;
  Arith a;
  // packed descriptors (host staging in pinned memory, same layout as the
  // workspace prefix starting at off_forms)
  char* staging = nullptr;
  size_t off_queue = 0, off_forms = 0, off_blobs = 0, off_leaves = 0, off_tables = 0, off_perms = 0, off_order = 0,
         off_results = 0, off_limbs = 0, off_arena = 0, total = 0;
  size_t desc_bytes = 0;
  uint32_t n_forms = 0;
  uint64_t total_out = 0;
  std::vector<uint64_t> res_off;
  uint64_t max_arena = 0;    // entries
  uint64_t max_blob = 0;     // bytes of the largest descriptor blob
  uint64_t slot_entries = 0;  // global arena slot of one CTA (entries)
  uint32_t slots = 0;         // CTAs any launch shape can have
  // launch configuration (autotuned)
  int threads = 128;
  int cta_cap = 0;           // CTAs per SM cap (0: as many as fit)
  size_t smem_bytes = 0;     // dynamic shared memory for arenas (per CTA), beyond the blob
  std::vector<int> grid;     // per residue group
  // graph cache
  cudaGraphExec_t gexec = nullptr;
  void* g_ws = nullptr;
  cudaStream_t g_stream = nullptr;
  ~tnc_batch_s() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (staging) cudaFreeHost(staging);
  }
};

namespace {

constexpr size_t kSmemMax = 227 * 1024;

// CTAs of batch_kernel<RG, N30> per SM for (threads, dynamic shared memory),
// capped at `cap` (0: no cap).  The L1 / shared-memory split is then set to
// the smallest shared-memory share that holds those CTAs, so that the rest of
// the SM's 256 KiB serves as L1 for the formulas' global arenas.
template <int RG, bool N30>
int occupancy(int threads, size_t smem, int cap, int* blocks) {
  auto k = tnc_dev::batch_kernel<RG, N30>;
  // the limit is a property of the kernel, shared by every batch in the
  // process: set it to the device's maximum, not to this batch's need (a batch
  // configured later with smaller descriptors would otherwise make an earlier
  // batch's launches fail)
  int optin = 0, dev0 = 0;
  cudaFuncAttributes fa{};
  CUDA_TRY(cudaGetDevice(&dev0));
  CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev0));
  CUDA_TRY(cudaFuncGetAttributes(&fa, k));
  const int dyn_max = optin - (int)fa.sharedSizeBytes;  // the opt-in limit covers static + dynamic
  if (smem > (size_t)std::max(dyn_max, 0))
    return set_error(TNC_ERR_TOO_LARGE, "batch kernel needs more shared memory than a CTA has");
  CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
  CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  int occ = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem));
  if (cap > 0) occ = std::min(occ, cap);
  int dev = 0, per_sm = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  if (occ > 0 && per_sm > 0) {
    const size_t need = (size_t)occ * (smem + 1024 + 64);
    const int pct = (int)std::min<size_t>(100, (need * 100 + per_sm - 1) / per_sm);
    CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    int occ2 = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k, threads, smem));
    if (occ2 < occ) CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  }
  *blocks = occ;
  return TNC_OK;
}

// Launch shape for (threads, smem, CTAs per SM cap) on every residue group.
int batch_configure(tnc_batch_t* b, int threads, size_t smem, int cap) {
  const int sms = sm_count();
  std::vector<int> grid;
  for (size_t gi = 0; gi < b->a.groups.rg.size(); gi++) {
    int occ = 0;
    const bool n30 = b->a.group((int)gi).near30 != 0;
    int rc = dispatch_rg(b->a.groups.rg[gi], [&](auto rgc) -> int {
      return n30 ? occupancy<decltype(rgc)::value, true>(threads, b->max_blob + smem, cap, &occ)
                 : occupancy<decltype(rgc)::value, false>(threads, b->max_blob + smem, cap, &occ);
    });
    if (rc) return rc;
    if (occ <= 0) return set_error(TNC_ERR_TOO_LARGE, "batch kernel does not fit on an SM");
    grid.push_back(std::max(1, std::min<int>(std::min<int>(sms * occ, (int)b->n_forms), (int)b->slots)));
  }
  b->threads = threads;
  b->smem_bytes = smem;
  b->cta_cap = cap;
  b->grid = grid;
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  return TNC_OK;
}

uint16_t pack_run(int src, int dst, int len) { return (uint16_t)(src | (dst << 5) | (len << 10)); }

// Appends `bytes` at a 16-byte boundary of the blob; returns the offset.
size_t blob_put(std::vector<char>& blob, const void* src, size_t bytes) {
  const size_t at = (blob.size() + 15) / 16 * 16;
  blob.resize(at + bytes);
  if (bytes) std::memcpy(blob.data() + at, src, bytes);
  return at;
}

int batch_pack(tnc_batch_t* b) {
  const uint32_t n = b->n_forms;
  std::vector<BForm> forms(n);
  std::vector<char> blobs;  // all formulas' blobs, each 16-byte aligned
  std::vector<BLeaf> leaves;
  std::vector<uint32_t> tables;
  std::vector<uint8_t> perms;
  b->res_off.assign(n, 0);
  uint64_t out = 0;
  b->max_arena = 8;
  b->max_blob = 16;
  for (uint32_t i = 0; i < n; i++) {
    const tnc_plan_t* p = b->plans[i];
    if (p->tree.nodes.empty()) return set_error(TNC_ERR_INVALID, "batch formula with an empty network");
    if (p->cost.max_rank > 24 || !p->low.lvl_fits)
      return set_error(TNC_ERR_TOO_LARGE, "batch formulas must have plan rank <= 24");
    const Lowered& lw = p->low;
    if (lw.lvl_arena_entries >= (1ull << 32)) return set_error(TNC_ERR_TOO_LARGE, "formula arena above 2^32 entries");
    if (lw.lvl_steps.size() >= 65535) return set_error(TNC_ERR_TOO_LARGE, "more than 65534 steps in one formula");
    // per level: the share of one lane of a 256-thread CTA (at least 16
    // products), and per step the lane split sh of its long shared sums: an
    // entry of a step is split over 2^sh lanes so that no lane sums much more
    // than that share
    const uint32_t nlev = lw.lvl_start.empty() ? 0 : (uint32_t)lw.lvl_start.size() - 1;
    std::vector<uint32_t> lvl_log_t(nlev, 4), step_sh(lw.lvl_steps.size(), 0);
    for (uint32_t l = 0; l < nlev; l++) {
      uint64_t work = 0;
      for (uint32_t si = lw.lvl_start[l]; si < lw.lvl_start[l + 1]; si++)
        work += 1ull << (lw.lvl_steps[si].c + lw.lvl_steps[si].k);
      uint32_t log_t = 4;
      while (log_t < 24 && (1ull << log_t) * 256 < work) log_t++;
      lvl_log_t[l] = log_t;
      for (uint32_t si = lw.lvl_start[l]; si < lw.lvl_start[l + 1]; si++) {
        const StepDesc& d = lw.lvl_steps[si];
        uint32_t sh = 0;
        while (sh < 5 && sh < d.k && d.k - sh > log_t) sh++;
        step_sh[si] = sh;
      }
    }
    // steps, runs and address deltas.  A lane group of a whole-warp block
    // advances its entry by 2^g (g = 5 - sh): delta[t - g] = w[t] -
    // sum_{g <= j < t} w[j] for the operand weights w[j] of output bit j.
    std::vector<BStep> steps;
    std::vector<uint16_t> runs;
    std::vector<int32_t> dls;  // pairs (A, B)
    for (size_t si = 0; si < lw.lvl_steps.size(); si++) {
      const StepDesc& d = lw.lvl_steps[si];
      BStep bs;
      std::memset(&bs, 0, sizeof(bs));
      bs.a_off = (uint32_t)d.a_off;
      bs.b_off = (uint32_t)d.b_off;
      bs.c_off = (uint32_t)d.c_off;
      bs.c = d.c;
      bs.k = d.k;
      bs.ka = d.ka;
      bs.kb = d.kb;
      if (runs.size() >= 65535 || dls.size() / 2 >= 65535)
        return set_error(TNC_ERR_TOO_LARGE, "formula descriptors beyond 2^16 runs or deltas");
      bs.run0 = (uint16_t)runs.size();
      int64_t wA[32] = {0}, wB[32] = {0};
      if (d.nra != TNC_BITMAP) {
        for (int r = 0; r < d.nra; r++) {
          const TncRun& x = d.map.runs.ra[r];
          runs.push_back(pack_run(x.src, x.dst, x.len));
          for (int q = 0; q < x.len; q++) wA[x.src + q] = 1ll << (x.dst + q);
        }
        for (int r = 0; r < d.nrb; r++) {
          const TncRun& x = d.map.runs.rb[r];
          runs.push_back(pack_run(x.src, x.dst, x.len));
          for (int q = 0; q < x.len; q++) wB[x.src + q] = 1ll << (x.dst + q);
        }
        bs.nra = d.nra;
        bs.nrb = d.nrb;
      } else {
        for (int side = 0; side < 2; side++)
          for (int j = 0; j < d.c; j++)
            if ((d.map.bit[j] >> 7) == side) {
              runs.push_back(pack_run(j, d.map.bit[j] & 63, 1));
              (side ? bs.nrb : bs.nra)++;
              (side ? wB : wA)[j] = 1ll << (d.map.bit[j] & 63);
            }
      }
      const uint32_t g = 5 - step_sh[si];
      bs.g = (uint8_t)g;
      bs.dl0 = (uint16_t)(dls.size() / 2);
      for (uint32_t t = g; t < d.c; t++) {
        int64_t sa = 0, sb = 0;
        for (uint32_t j = g; j < t; j++) {
          sa += wA[j];
          sb += wB[j];
        }
        dls.push_back((int32_t)(wA[t] - sa));
        dls.push_back((int32_t)(wB[t] - sb));
      }
      steps.push_back(bs);
    }
    // segments per level: steps whose entries take 32+ lanes get whole-warp
    // blocks of V entries per lane group (V such that a lane's work is about
    // half the level's share, at most 4); the others share packed segments
    // lane by lane.  Segments are ordered by cost, longest first.
    std::vector<Seg> segs;
    std::vector<uint32_t> items, lvl{0};
    for (uint32_t l = 0; l < nlev; l++) {
      const uint32_t log_t = lvl_log_t[l];
      struct Group {
        uint32_t si, o, sh, cost;
      };
      std::vector<Group> small;
      std::vector<std::pair<uint32_t, Seg>> lsegs;  // (cost, segment)
      for (uint32_t si = lw.lvl_start[l]; si < lw.lvl_start[l + 1]; si++) {
        const StepDesc& d = lw.lvl_steps[si];
        const uint32_t sh = step_sh[si];
        const uint32_t cost = 1u << (d.k - sh);
        const uint32_t nout = 1u << d.c;
        if ((nout << sh) < 32) {
          for (uint32_t o = 0; o < nout; o++) small.push_back(Group{si, o, sh, cost});
          continue;
        }
        const uint32_t G = 32u >> sh;
        uint32_t V = 1;
        while (V < 4 && 2 * V * G <= nout && (2 * V) * cost <= (1u << (log_t - 1))) V *= 2;
        for (uint32_t o0 = 0; o0 < nout; o0 += G * V)
          lsegs.push_back({cost * V, Seg{o0, (uint16_t)si, (uint8_t)V, (uint8_t)sh}});
      }
      // widest groups first: each group then starts at a multiple of its size
      // and never crosses a 32-lane boundary
      std::stable_sort(small.begin(), small.end(), [](const Group& x, const Group& y) {
        return x.sh != y.sh ? x.sh > y.sh : x.cost > y.cost;
      });
      for (size_t g = 0; g < small.size();) {
        const uint32_t first = (uint32_t)items.size();
        uint32_t lanes = 0, cost = 0;
        const uint8_t sh0 = (uint8_t)small[g].sh;
        while (g < small.size() && lanes + (1u << small[g].sh) <= 32) {
          const Group& q = small[g];
          for (uint32_t j = 0; j < (1u << q.sh); j++) items.push_back(q.si | q.o << 16 | j << 21 | q.sh << 26);
          lanes += 1u << q.sh;
          cost = std::max(cost, q.cost);
          g++;
        }
        lsegs.push_back({cost, Seg{first, tnc_dev::kPacked, (uint8_t)lanes, sh0}});
      }
      std::stable_sort(lsegs.begin(), lsegs.end(),
                       [](const std::pair<uint32_t, Seg>& x, const std::pair<uint32_t, Seg>& y) {
                         return x.first > y.first;
                       });
      for (const auto& x : lsegs) segs.push_back(x.second);
      lvl.push_back((uint32_t)segs.size());
    }
    // the blob
    std::vector<char> blob;
    blob_put(blob, steps.data(), steps.size() * sizeof(BStep));
    BForm& f = forms[i];
    std::memset(&f, 0, sizeof(f));
    f.segs_at = (uint32_t)blob_put(blob, segs.data(), segs.size() * sizeof(Seg));
    f.items_at = (uint32_t)blob_put(blob, items.data(), items.size() * sizeof(uint32_t));
    f.runs_at = (uint32_t)blob_put(blob, runs.data(), runs.size() * sizeof(uint16_t));
    f.dl_at = (uint32_t)blob_put(blob, dls.data(), dls.size() * sizeof(int32_t));
    f.lvl_at = (uint32_t)blob_put(blob, lvl.data(), lvl.size() * sizeof(uint32_t));
    blob.resize((blob.size() + 15) / 16 * 16);
    f.blob = (uint32_t)(blobs.size() / 16);
    f.blob_n = (uint32_t)(blob.size() / 16);
    blobs.insert(blobs.end(), blob.begin(), blob.end());
    b->max_blob = std::max<uint64_t>(b->max_blob, blob.size());
    f.nlev = nlev;
    f.leaf0 = (uint32_t)leaves.size();
    f.nleaf = (uint32_t)lw.leaves.size();
    f.res_off = (uint32_t)out;
    f.n_open = (uint32_t)p->net.open_vars.size();
    f.n_out = 1u << f.n_open;
    f.perm_off = (uint32_t)perms.size();
    f.root_off = (uint32_t)(lw.lvl_steps.empty() ? lw.lvl_leaf_off[p->tree.root] : lw.lvl_root_off);
    f.arena = (uint32_t)lw.lvl_arena_entries;

    b->res_off[i] = out;
    out += f.n_out;
    const uint32_t toff = (uint32_t)tables.size();
    for (size_t l = 0; l < lw.leaves.size(); l++) {
      BLeaf bl;
      std::memset(&bl, 0, sizeof(bl));
      bl.off = (uint32_t)lw.lvl_leaf_off[l];
      bl.table_off = lw.leaves[l].table_off + toff;
      bl.kind = lw.leaves[l].kind;
      bl.rank = lw.leaves[l].rank;
      leaves.push_back(bl);
    }
    tables.insert(tables.end(), lw.leaf_tables.begin(), lw.leaf_tables.end());
    perms.insert(perms.end(), lw.root_perm.begin(), lw.root_perm.end());
    b->max_arena = std::max<uint64_t>(b->max_arena, lw.lvl_arena_entries);
  }
  if (blobs.size() / 16 >= (1ull << 32)) return set_error(TNC_ERR_TOO_LARGE, "batch descriptors above 64 GiB");
  b->total_out = out;
  // one global arena slot per CTA: at most 32 CTAs per SM in any launch shape
  b->slot_entries = (b->max_arena + 7) / 8 * 8;
  b->slots = (uint32_t)std::min<uint64_t>(n, (uint64_t)sm_count() * 32u);
  // largest formulas first (longest-processing-time order)
  std::vector<uint32_t> order(n);
  for (uint32_t i = 0; i < n; i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
    return b->plans[x]->cost.macs + b->plans[x]->cost.entries > b->plans[y]->cost.macs + b->plans[y]->cost.entries;
  });
  const int rg_max = b->a.groups.rg.empty() ? 1 : b->a.groups.rg[0];
  // workspace layout
  size_t o = 0;
  auto sect = [&](size_t& off, size_t bytes) {
    off = o;
    o = align_up(o + bytes);
  };
  sect(b->off_queue, 64 * sizeof(uint32_t));
  sect(b->off_forms, forms.size() * sizeof(BForm));
  sect(b->off_blobs, blobs.size());
  sect(b->off_leaves, leaves.size() * sizeof(BLeaf));
  sect(b->off_tables, tables.size() * sizeof(uint32_t));
  sect(b->off_perms, perms.size());
  sect(b->off_order, order.size() * sizeof(uint32_t));
  b->desc_bytes = o - b->off_forms;
  sect(b->off_results, out * b->a.R * sizeof(uint32_t));
  sect(b->off_limbs, out * b->a.crt.n_limbs * sizeof(uint32_t));
  sect(b->off_arena, (size_t)b->slots * b->slot_entries * rg_max * sizeof(uint32_t));
  b->total = o;
  CUDA_TRY(cudaMallocHost((void**)&b->staging, std::max<size_t>(b->desc_bytes, 1)));
  std::memset(b->staging, 0, b->desc_bytes);
  char* s = b->staging - b->off_forms;
  auto put = [&](size_t off, const void* src, size_t bytes) {
    if (bytes) std::memcpy(s + off, src, bytes);
  };
  put(b->off_forms, forms.data(), forms.size() * sizeof(BForm));
  put(b->off_blobs, blobs.data(), blobs.size());
  put(b->off_leaves, leaves.data(), leaves.size() * sizeof(BLeaf));
  put(b->off_tables, tables.data(), tables.size() * sizeof(uint32_t));
  put(b->off_perms, perms.data(), perms.size());
  put(b->off_order, order.data(), order.size() * sizeof(uint32_t));
  // default launch shape (the autotuner's usual pick): 256 threads, arenas in
  // global memory, as many CTAs per SM as fit
  if (b->max_blob > kSmemMax) return set_error(TNC_ERR_TOO_LARGE, "a formula's descriptors exceed shared memory");
  return batch_configure(b, 256, 0, 0);
}

int batch_enqueue(tnc_batch_t* b, void* dev_ws, cudaStream_t st) {
  char* ws = (char*)dev_ws;
  CUDA_TRY(cudaMemsetAsync(ws + b->off_queue, 0, 64 * sizeof(uint32_t), st));
  for (size_t gi = 0; gi < b->a.groups.rg.size(); gi++) {
    const int rg = b->a.groups.rg[gi];
    BatchArgs args{};
    args.forms = (const BForm*)(ws + b->off_forms);
    args.blobs = (const uint4*)(ws + b->off_blobs);
    args.leaves = (const BLeaf*)(ws + b->off_leaves);
    args.tables = (const uint32_t*)(ws + b->off_tables);
    args.perms = (const uint8_t*)(ws + b->off_perms);
    args.order = (const uint32_t*)(ws + b->off_order);
    args.n_forms = b->n_forms;
    args.queue = (uint32_t*)(ws + b->off_queue) + gi;
    args.results = (uint32_t*)(ws + b->off_results);
    args.garena = (uint32_t*)(ws + b->off_arena);
    args.slot_entries = b->slot_entries;
    args.blob_cap = (uint32_t)b->max_blob;
    args.smem_cap = (uint32_t)(b->smem_bytes / (rg * sizeof(uint32_t)));
    args.R = b->a.R;
    args.col = b->a.groups.col[gi];
    const ModGroup mg = b->a.group((int)gi);
    const int grid = b->grid[gi];
    const size_t smem = b->max_blob + b->smem_bytes;
    const int threads = b->threads;
    int rc = dispatch_rg(rg, [&](auto rgc) -> int {
      constexpr int RG = decltype(rgc)::value;
      if (mg.near30) tnc_dev::batch_kernel<RG, true><<<grid, threads, smem, st>>>(args, mg);
      else tnc_dev::batch_kernel<RG, false><<<grid, threads, smem, st>>>(args, mg);
      CUDA_TRY(cudaGetLastError());
      return TNC_OK;
    });
    if (rc) return rc;
  }
  tnc_dev::crt_kernel<<<(unsigned)std::max<uint64_t>(1, std::min<uint64_t>((b->total_out + 127) / 128, 4096)), 128, 0,
                        st>>>((const uint32_t*)(ws + b->off_results), b->total_out, b->a.crt,
                              (uint32_t*)(ws + b->off_limbs));
  CUDA_TRY(cudaGetLastError());
  return TNC_OK;
}

}  // namespace

extern "C" int tnc_batch_create(const tnc_plan_t* const* plans, int32_t n, const tnc_contract_opts* opts,
                                tnc_batch_t** out) {
  clear_error();
  if (!plans || n <= 0 || !out) return set_error(TNC_ERR_INVALID, "bad batch arguments");
  *out = nullptr;
  try {
    if (inject_hit(TNC_INJECT_NOMEM)) throw std::bad_alloc();
    auto* b = new tnc_batch_t();
    int rc = make_arith(opts, b->a);
    if (!rc && opts->path == TNC_PATH_TC_P8)
      rc = set_error(TNC_ERR_INVALID, "TNC_PATH_TC_P8 is a tnc_contract path; batches run TNC_PATH_INT64");
    if (!rc) {
      for (int i = 0; i < n; i++) {
        if (!plans[i]) rc = set_error(TNC_ERR_INVALID, "NULL plan in batch");
        b->plans.push_back(plans[i]);
      }
    }
    b->n_forms = (uint32_t)n;
    if (!rc) rc = batch_pack(b);
    if (rc) {
      delete b;
      return rc;
    }
    *out = b;
    return TNC_OK;
  } catch (const std::bad_alloc&) {
    return set_error(TNC_ERR_NOMEM, "out of host memory");
  }
}

extern "C" size_t tnc_batch_workspace_bytes(const tnc_batch_t* b) { return b ? b->total : 0; }

extern "C" int tnc_batch_info(const tnc_batch_t* b, size_t* h2d_bytes, size_t* d2h_bytes, uint64_t* n_entries,
                              int32_t* kernels_per_launch) {
  clear_error();
  if (!b) return set_error(TNC_ERR_INVALID, "batch is NULL");
  if (h2d_bytes) *h2d_bytes = b->desc_bytes;
  if (d2h_bytes) *d2h_bytes = b->total_out * (size_t)(b->a.R + b->a.crt.n_limbs) * sizeof(uint32_t);
  if (n_entries) *n_entries = b->total_out;
  if (kernels_per_launch) *kernels_per_launch = (int32_t)b->a.groups.rg.size() + 1;
  return TNC_OK;
}

extern "C" int tnc_batch_upload(tnc_batch_t* b, void* dev_ws, size_t ws_bytes, void* cuda_stream) {
  clear_error();
  if (!b || !dev_ws) return set_error(TNC_ERR_INVALID, "NULL argument");
  if (ws_bytes < b->total) return set_error(TNC_ERR_BUFFER, "workspace smaller than tnc_batch_workspace_bytes");
  if (((uintptr_t)dev_ws) % kAlign) return set_error(TNC_ERR_INVALID, "workspace must be 256-byte aligned");
  CUDA_TRY(cudaMemcpyAsync((char*)dev_ws + b->off_forms, b->staging, b->desc_bytes, cudaMemcpyHostToDevice,
                           (cudaStream_t)cuda_stream));
  return TNC_OK;
}

extern "C" int tnc_batch_launch(tnc_batch_t* b, void* dev_ws, void* cuda_stream) {
  clear_error();
  if (!b || !dev_ws) return set_error(TNC_ERR_INVALID, "NULL argument");
  if (inject_hit(TNC_INJECT_LAUNCH)) return set_error(TNC_ERR_CUDA, "injected failure (TNC_INJECT_LAUNCH)");
  NvtxRange range("tnc_batch_launch");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (st == nullptr) return batch_enqueue(b, dev_ws, st);  // legacy stream: cannot capture
  if (b->gexec && (b->g_ws != dev_ws || b->g_stream != st)) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  if (!b->gexec) {
    CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = batch_enqueue(b, dev_ws, st);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return set_error(TNC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->gexec = nullptr;
      return set_error(TNC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    b->g_ws = dev_ws;
    b->g_stream = st;
  }
  CUDA_TRY(cudaGraphLaunch(b->gexec, st));
  return TNC_OK;
}

extern "C" int tnc_batch_autotune(tnc_batch_t* b, void* dev_ws, void* cuda_stream, int32_t* threads_out,
                                  int32_t* smem_out, int32_t* ctas_out) {
  clear_error();
  if (!b || !dev_ws) return set_error(TNC_ERR_INVALID, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int rg_max = b->a.groups.rg.empty() ? 1 : b->a.groups.rg[0];
  const size_t need = b->max_arena * rg_max * sizeof(uint32_t);
  std::vector<size_t> smems{0};
  for (size_t s : {16u << 10, 32u << 10, 48u << 10, 64u << 10, 96u << 10, 128u << 10, 192u << 10})
    if (s + b->max_blob <= kSmemMax) smems.push_back(std::min(s, need));
  std::sort(smems.begin(), smems.end());
  smems.erase(std::unique(smems.begin(), smems.end()), smems.end());
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_t = b->threads, best_c = b->cta_cap;
  size_t best_s = b->smem_bytes;
  int rc = TNC_OK;
  for (int threads : {64, 128, 256}) {
    for (size_t sm : smems) {
      int prev_grid = -1;
      for (int cap : {0, 2, 1}) {
        rc = batch_configure(b, threads, sm, cap);
        if (rc == TNC_ERR_TOO_LARGE) {
          rc = TNC_OK;
          break;
        }
        if (rc) break;
        if (b->grid[0] == prev_grid) continue;  // the cap changes nothing
        prev_grid = b->grid[0];
        float ms = 1e30f;
        for (int rep = 0; rep < 2 && !rc; rep++) {
          cudaEventRecord(e0, st);
          rc = batch_enqueue(b, dev_ws, st);
          cudaEventRecord(e1, st);
          if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = set_error(TNC_ERR_CUDA, "autotune launch failed");
          float t = 0;
          if (!rc) cudaEventElapsedTime(&t, e0, e1);
          if (rep == 1) ms = t;
        }
        if (rc) break;
        if (ms < best) {
          best = ms;
          best_t = threads;
          best_s = sm;
          best_c = cap;
        }
      }
      if (rc) break;
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  rc = batch_configure(b, best_t, best_s, best_c);
  if (threads_out) *threads_out = best_t;
  if (smem_out) *smem_out = (int32_t)best_s;
  if (ctas_out) *ctas_out = best_c;
  return rc;
}

extern "C" int tnc_batch_set_launch(tnc_batch_t* b, int32_t threads, int32_t smem_bytes, int32_t ctas_per_sm) {
  clear_error();
  if (!b) return set_error(TNC_ERR_INVALID, "NULL argument");
  if (threads != 64 && threads != 128 && threads != 256)
    return set_error(TNC_ERR_INVALID, "threads must be 64, 128 or 256");
  if (ctas_per_sm < 0) return set_error(TNC_ERR_INVALID, "ctas_per_sm must be >= 0");
  if (smem_bytes < 0 || (size_t)smem_bytes + b->max_blob > kSmemMax)
    return set_error(TNC_ERR_TOO_LARGE, "shared-memory arena too large");
  return batch_configure(b, threads, (size_t)smem_bytes, ctas_per_sm);
}

extern "C" int tnc_batch_get_launch(const tnc_batch_t* b, int32_t* threads, int32_t* smem_bytes,
                                    int32_t* ctas_per_sm) {
  clear_error();
  if (!b) return set_error(TNC_ERR_INVALID, "NULL argument");
  if (threads) *threads = b->threads;
  if (smem_bytes) *smem_bytes = (int32_t)b->smem_bytes;
  if (ctas_per_sm) *ctas_per_sm = b->cta_cap;
  return TNC_OK;
}

extern "C" int tnc_batch_download(tnc_batch_t* b, const void* dev_ws, void* cuda_stream, tnc_count* outs) {
  clear_error();
  if (!b || !dev_ws || !outs) return set_error(TNC_ERR_INVALID, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::vector<uint32_t> res(b->total_out * b->a.R), limbs(b->total_out * b->a.crt.n_limbs);
  CUDA_TRY(cudaMemcpyAsync(res.data(), (const char*)dev_ws + b->off_results, res.size() * 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(limbs.data(), (const char*)dev_ws + b->off_limbs, limbs.size() * 4, cudaMemcpyDeviceToHost,
                           st));
  CUDA_TRY(cudaStreamSynchronize(st));
  for (uint32_t i = 0; i < b->n_forms; i++) {
    const tnc_plan_t* p = b->plans[i];
    const uint64_t n_out = 1ull << p->net.open_vars.size();
    int rc = fill_count(&outs[i], n_out, b->a, res.data() + b->res_off[i] * b->a.R,
                        limbs.data() + b->res_off[i] * b->a.crt.n_limbs, result_flags(p, b->a));
    if (rc) return rc;
  }
  return TNC_OK;
}

extern "C" int tnc_batch_download_flat(tnc_batch_t* b, const void* dev_ws, void* cuda_stream, uint32_t* residues,
                                       uint32_t* limbs, uint32_t* flags) {
  clear_error();
  if (!b || !dev_ws) return set_error(TNC_ERR_INVALID, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (residues)
    CUDA_TRY(cudaMemcpyAsync(residues, (const char*)dev_ws + b->off_results, b->total_out * b->a.R * sizeof(uint32_t),
                             cudaMemcpyDeviceToHost, st));
  if (limbs)
    CUDA_TRY(cudaMemcpyAsync(limbs, (const char*)dev_ws + b->off_limbs,
                             b->total_out * b->a.crt.n_limbs * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  if (flags)
    for (uint32_t i = 0; i < b->n_forms; i++) flags[i] = result_flags(b->plans[i], b->a);
  CUDA_TRY(cudaStreamSynchronize(st));
  return TNC_OK;
}

extern "C" int tnc_batch_status(tnc_batch_t* b, const void* dev_ws, void* cuda_stream) {
  clear_error();
  if (!b || !dev_ws) return set_error(TNC_ERR_INVALID, "NULL argument");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)cuda_stream));
  return TNC_OK;
}

extern "C" void tnc_free_batch(tnc_batch_t* b) { delete b; }

extern "C" int tnc_contract_batch(const tnc_plan_t* const* plans, int32_t n, const tnc_contract_opts* opts, void* dev_ws,
                                  size_t ws_bytes, void* cuda_stream, tnc_count* outs) {
  tnc_batch_t* b = nullptr;
  int rc = tnc_batch_create(plans, n, opts, &b);
  if (rc) return rc;
  rc = tnc_batch_upload(b, dev_ws, ws_bytes, cuda_stream);
  if (!rc) rc = batch_enqueue(b, dev_ws, (cudaStream_t)cuda_stream);
  if (!rc) rc = tnc_batch_download(b, dev_ws, cuda_stream, outs);
  tnc_free_batch(b);
  return rc;
}

// =============================================== allocation-free single formula
//
// For callers that must not allocate device memory (see tnc_contract_noalloc
// in tnc.h).  All device scratch -- leaf descriptors, weight tables, step
// descriptors, the tensor arena, residues and CRT limbs -- lives in one
// file-scope array that every GPU loading this library holds until exit.
// Nothing in the path needs it to start zeroed: the leaf fill writes every
// leaf entry, every step writes each output entry before any later step
// reads it, and the residue and limb regions are written in full.  Host-side
// work uses fixed-size stack buffers only.

static __device__ __align__(256) unsigned char g_noalloc_scratch[TNC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_base[kMaxDevices] = {nullptr};
CUcontext g_noalloc_ctx[kMaxDevices] = {nullptr};

// The driver's current context, fetched through the runtime (no link-time
// dependency on the driver library); nullptr if unavailable.
CUcontext current_context() {
  using GetCtx = CUresult (*)(CUcontext*);
  static GetCtx fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<GetCtx>(p);
  }();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// Device address of the scratch array on the current device.  In host code
// `g_noalloc_scratch` names a host-side shadow, not device memory, so the
// address is looked up once per device, with that device current, and kept
// with the context it belongs to: after a device reset the runtime makes a
// new context (and loads the module again), and the address is looked up
// anew.  (Before the runtime has made a context current the context reads as
// nullptr; the next call then looks the address up once more.)
int noalloc_base(void** out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(TNC_ERR_INVALID, "device ordinal out of range");
  const CUcontext ctx = current_context();
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_base[dev] || g_noalloc_ctx[dev] != ctx) {
    void* p = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    if (!p) return set_error(TNC_ERR_CUDA, "cudaGetSymbolAddress returned NULL");
    g_noalloc_base[dev] = p;
    g_noalloc_ctx[dev] = ctx;
  }
  *out = g_noalloc_base[dev];
  return TNC_OK;
}

}  // namespace

extern "C" int tnc_contract_noalloc(const tnc_plan_t* plan, const tnc_contract_opts* opts, void* cuda_stream,
                                    tnc_count* out) {
  clear_error();
  g_launches = tnc_launch_counts{};
  NvtxRange range("tnc_contract_noalloc");
  if (!plan || !opts || !out) return set_error(TNC_ERR_INVALID, "NULL argument");
  if (opts->path != TNC_PATH_INT64)
    return set_error(TNC_ERR_INVALID, "tnc_contract_noalloc supports TNC_PATH_INT64 only");
  const int R = opts->n_residues;
  if (R < 1 || R > 16) return set_error(TNC_ERR_INVALID, "n_residues must be in [1, 16]");
  // primes and CRT constants, on the stack
  uint32_t primes[16];
  if (opts->primes) {
    for (int i = 0; i < R; i++) {
      const uint32_t p = opts->primes[i];
      if (p <= (1u << 29) || p >= (1u << 31) || !is_prime_u32(p))
        return set_error(TNC_ERR_INVALID, "primes must be primes in (2^29, 2^31)");
      for (int j = 0; j < i; j++)
        if (primes[j] == p) return set_error(TNC_ERR_INVALID, "primes must be distinct");
      primes[i] = p;
    }
  } else {
    int n = 0;
    for (uint32_t x = kDefaultPrimeBound - 1; n < R; x -= 2)
      if (is_prime_u32(x)) primes[n++] = x;
  }
  CrtConsts cc{};
  cc.R = R;
  double log2_prod = 0;
  for (int i = 0; i < R; i++) {
    const uint32_t p = primes[i];
    cc.p[i] = p;
    cc.mu[i] = ~0ull / p;
    uint64_t prod = 1;
    for (int j = 0; j < i; j++) prod = prod * (primes[j] % p) % p;
    cc.inv[i] = i == 0 ? 1u : powmod(prod, p - 2, p);
    log2_prod += std::log2((double)p);
  }
  cc.n_limbs = (31 * R + 31) / 32;
  int n_groups = 0, grp_rg[16], grp_col[16];
  for (int c = 0, s = 4; s >= 1; s /= 2)
    while (R - c >= s) {
      grp_rg[n_groups] = s;
      grp_col[n_groups++] = c;
      c += s;
    }

  const SeqLayout L = seq_layout(plan, R);
  const uint64_t n_out = L.n_out;
  out->n_out = (int32_t)n_out;
  out->n_limbs = cc.n_limbs;
  out->flags = plan->net.log2_bound >= log2_prod - 1e-9 ? TNC_MAYBE_WRAPPED : 0u;
  if (out->cap_out < (int32_t)n_out) return set_error(TNC_ERR_BUFFER, "count buffer holds fewer entries than 2^n_open");
  if (out->limbs && out->cap_limbs < cc.n_limbs)
    return set_error(TNC_ERR_BUFFER, "need " + std::to_string(cc.n_limbs) + " limbs");
  if (plan->tree.nodes.empty()) {  // empty network: the empty product, 1
    out->flags = 0;
    if (out->residues)
      for (int r = 0; r < R; r++) out->residues[r] = 1u;
    if (out->limbs) {
      std::memset(out->limbs, 0, (size_t)out->cap_limbs * sizeof(uint32_t));
      out->limbs[0] = 1u;
    }
    return TNC_OK;
  }
  if (L.total > (size_t)TNC_NOALLOC_SCRATCH_BYTES)
    return set_error(TNC_ERR_TOO_LARGE, "plan needs " + std::to_string(L.total) +
                                            " bytes of scratch; tnc_contract_noalloc holds " +
                                            std::to_string((size_t)TNC_NOALLOC_SCRATCH_BYTES));
  if (inject_hit(TNC_INJECT_LAUNCH)) return set_error(TNC_ERR_CUDA, "injected failure (TNC_INJECT_LAUNCH)");
  void* base = nullptr;
  int rc = noalloc_base(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  char* ws = (char*)base;

  // descriptors: through small stack buffers (pageable copies return once the
  // source has been staged, so the buffer can be refilled right away)
  {
    LeafDesc buf[64];
    const size_t nl = plan->low.leaves.size();
    for (size_t i0 = 0; i0 < nl; i0 += 64) {
      const size_t m = std::min<size_t>(64, nl - i0);
      for (size_t i = 0; i < m; i++) {
        buf[i] = plan->low.leaves[i0 + i];
        buf[i].off = plan->low.seq_leaf_off[i0 + i];
      }
      CUDA_TRY(cudaMemcpyAsync(ws + L.off_leaves + i0 * sizeof(LeafDesc), buf, m * sizeof(LeafDesc),
                               cudaMemcpyHostToDevice, st));
    }
  }
  if (!plan->low.leaf_tables.empty())
    CUDA_TRY(cudaMemcpyAsync(ws + L.off_tables, plan->low.leaf_tables.data(),
                             plan->low.leaf_tables.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
  {
    GridStep buf[8];
    const size_t ns = plan->low.seq_steps.size();
    for (size_t i0 = 0; i0 < ns; i0 += 8) {
      const size_t m = std::min<size_t>(8, ns - i0);
      for (size_t i = 0; i < m; i++) buf[i] = make_grid_step(plan->low.seq_steps[i0 + i]);
      CUDA_TRY(cudaMemcpyAsync(ws + L.off_steps + i0 * sizeof(GridStep), buf, m * sizeof(GridStep),
                               cudaMemcpyHostToDevice, st));
    }
  }
  const GridStep* d_steps = (const GridStep*)(ws + L.off_steps);
  uint32_t* arena = (uint32_t*)(ws + L.off_arena);
  uint32_t* results = (uint32_t*)(ws + L.off_results);
  uint32_t* limbs = (uint32_t*)(ws + L.off_limbs);
  uint32_t* part = (uint32_t*)(ws + L.off_part);
  RootMap rm{};
  rm.n_open = (int)plan->net.open_vars.size();
  for (int j = 0; j < rm.n_open; j++) rm.perm[j] = plan->low.root_perm[j];
  const int nl = (int)plan->low.leaves.size();
  const int sms = sm_count();
  const uint64_t root_off =
      plan->low.seq_steps.empty() ? plan->low.seq_leaf_off[plan->tree.root] : plan->low.seq_root_off;
  for (int gi = 0; gi < n_groups; gi++) {
    uint32_t gp[4];
    for (int r = 0; r < 4; r++) gp[r] = r < grp_rg[gi] ? primes[grp_col[gi] + r] : primes[grp_col[gi]];
    const ModGroup mg = tnc_dev::make_mod_group(gp);
    rc = dispatch_rg(grp_rg[gi], [&](auto rgc) -> int {
      constexpr int RG = decltype(rgc)::value;
      tnc_dev::leaf_fill_kernel<RG><<<std::min(nl, sms * 8), 64, 0, st>>>(
          (const LeafDesc*)(ws + L.off_leaves), nl, (const uint32_t*)(ws + L.off_tables), arena, mg);
      g_launches.leaf_fill++;
      for (size_t i = 0; i < plan->low.seq_steps.size(); i++) {
        const StepDesc& d = plan->low.seq_steps[i];
        const uint32_t ls = splitk_log(d);
        if (ls > 0) {  // few outputs, long shared sum: K split over blocks, as in tnc_contract
          tnc_dev::splitk_partial_kernel<RG><<<(unsigned)(1ull << (d.c + ls)), 256, 0, st>>>(d_steps + i, arena, part,
                                                                                           ls, mg);
          tnc_dev::splitk_final_kernel<RG><<<(unsigned)(1ull << d.c), 256, 0, st>>>(d_steps + i, arena, part, ls, mg);
          g_launches.splitk++;
          continue;
        }
        int threads, blocks, sh;
        grid_shape(d.c, &threads, &blocks, &sh);
        tnc_dev::step_kernel<RG><<<blocks, threads, 0, st>>>(d_steps + i, arena, mg);
        g_launches.grid_step++;
      }
      tnc_dev::extract_kernel<RG><<<(unsigned)std::min<uint64_t>((n_out + 255) / 256, 1024), 256, 0, st>>>(
          arena, root_off, rm, results, R, grp_col[gi]);
      g_launches.extract++;
      CUDA_TRY(cudaGetLastError());
      return TNC_OK;
    });
    if (rc) return rc;
  }
  tnc_dev::crt_kernel<<<(unsigned)std::min<uint64_t>((n_out + 127) / 128, 1024), 128, 0, st>>>(results, n_out, cc,
                                                                                                limbs);
  g_launches.crt++;
  CUDA_TRY(cudaGetLastError());
  if (out->residues)
    CUDA_TRY(cudaMemcpyAsync(out->residues, results, n_out * R * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  if (out->limbs) {
    std::memset(out->limbs, 0, n_out * (size_t)out->cap_limbs * sizeof(uint32_t));
    CUDA_TRY(cudaMemcpy2DAsync(out->limbs, (size_t)out->cap_limbs * sizeof(uint32_t), limbs,
                               (size_t)cc.n_limbs * sizeof(uint32_t), (size_t)cc.n_limbs * sizeof(uint32_t), n_out,
                               cudaMemcpyDeviceToHost, st));
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  return TNC_OK;
}

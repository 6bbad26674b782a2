// Lowering of a contraction tree to device descriptors.
//
// Every bond has dimension 2 (Sec. 2.1), so a tensor of rank r is a flat array
// of 2^r entries whose index bits are its bonds in a chosen order (its
// layout).  The permute + reshape-to-matrix of a pairwise step (Sec. 2.1,
// Corollary 2) then reduces to bit maps, and since the layout of every
// intermediate is free, it is chosen top-down so that each step reads its
// operands as plain matrices: operand X of the step that makes Z is laid out
// as [bonds X passes on to Z, in Z's order][bonds shared with the sibling],
// i.e. an M x K matrix with M contiguous.  The output index o of the step is
// then a few contiguous runs of A's and B's free bits.
#include <algorithm>
#include <cstring>
#include <map>

#include "tnc_internal.h"

namespace tnc {

// Interval allocation: tensors live over [t0, t1] (inclusive); two tensors
// whose lifetimes overlap never share memory.  First fit in t0 order; offsets
// are multiples of `align` entries.
static uint64_t allocate(const std::vector<uint64_t>& size, const std::vector<int>& t0,
                         const std::vector<int>& t1, std::vector<uint64_t>& off, uint64_t align = 8) {
  const size_t n = size.size();
  std::vector<int> ord(n);
  for (size_t i = 0; i < n; i++) ord[i] = (int)i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    return t0[a] != t0[b] ? t0[a] < t0[b] : size[a] > size[b];
  });
  off.assign(n, 0);
  std::vector<int> active;
  uint64_t peak = 0;
  for (int i : ord) {
    active.erase(std::remove_if(active.begin(), active.end(), [&](int a) { return t1[a] < t0[i]; }),
                 active.end());
    std::sort(active.begin(), active.end(), [&](int a, int b) { return off[a] < off[b]; });
    uint64_t need = (size[i] + align - 1) / align * align;
    uint64_t pos = 0;
    for (int a : active) {
      if (off[a] >= pos + need) break;
      uint64_t end = (off[a] + size[a] + align - 1) / align * align;
      pos = std::max(pos, end);
    }
    off[i] = pos;
    peak = std::max(peak, pos + need);
    active.push_back(i);
  }
  return peak;
}

int lower_plan(const Network& net, const Tree& tree, Lowered& low) {
  const int L = tree.n_leaves;
  const int N = (int)tree.nodes.size();
  low = Lowered();
  low.layout.assign(N, {});
  if (N == 0) return TNC_OK;
  const int root = tree.root;
  if (root < 0) return set_error(TNC_ERR_INVALID, "tree has no root");

  // Global bond order.  Bond b is contracted at node cnode(b) (where its two
  // ends meet); every tensor lists its bonds sorted by
  //   (depth of cnode(b), leaf DFS position of b's first end, b)
  // so the bonds a tensor's parent step contracts are its top bits (the K
  // block, in the same order in both operands), bonds contracted further up
  // sit lower, and any two tensors order their common bonds alike.  An output
  // index o therefore maps monotonically onto each operand's free bits.
  std::vector<int> depth(N, 0), parent(N, -1);
  for (int z = L; z < N; z++) {
    parent[tree.nodes[z].left] = z;
    parent[tree.nodes[z].right] = z;
  }
  for (int z = N - 1; z >= 0; z--)
    if (parent[z] >= 0) depth[z] = depth[parent[z]] + 1;
  std::vector<int> dfs(N, 0);
  {
    int pos = 0;
    std::vector<int> st{root};
    while (!st.empty()) {
      int u = st.back();
      st.pop_back();
      if (u < L) {
        dfs[u] = pos++;
        continue;
      }
      st.push_back(tree.nodes[u].right);
      st.push_back(tree.nodes[u].left);
    }
  }
  std::vector<int> cdepth(net.n_bonds, -1), first(net.n_bonds, 0);
  for (int z = L; z < N; z++) {
    const auto& lb = tree.nodes[tree.nodes[z].left].bonds;
    const auto& rb = tree.nodes[tree.nodes[z].right].bonds;
    std::vector<int> S;
    std::set_intersection(lb.begin(), lb.end(), rb.begin(), rb.end(), std::back_inserter(S));
    for (int b : S) cdepth[b] = depth[z];
  }
  for (int b = 0; b < net.n_bonds; b++) {
    int e0 = net.bond_end0[b], e1 = net.bond_end1[b];
    first[b] = e1 < 0 ? dfs[e0] : std::min(dfs[e0], dfs[e1]);
  }
  auto key_less = [&](int a, int b) {
    if (cdepth[a] != cdepth[b]) return cdepth[a] < cdepth[b];
    if (first[a] != first[b]) return first[a] < first[b];
    return a < b;
  };
  for (int i = 0; i < N; i++) {
    low.layout[i] = tree.nodes[i].bonds;
    std::sort(low.layout[i].begin(), low.layout[i].end(), key_less);
  }

  std::vector<StepDesc> desc(N);
  for (int z = L; z < N; z++) {
    const int x = tree.nodes[z].left, y = tree.nodes[z].right;
    const auto& lx = low.layout[x];
    const auto& ly = low.layout[y];
    const auto& lz = low.layout[z];
    StepDesc& d = desc[z];
    std::memset(&d, 0, sizeof(d));
    d.c = (uint8_t)lz.size();
    d.a_rank = (uint8_t)lx.size();
    d.b_rank = (uint8_t)ly.size();
    d.k = (uint8_t)((lx.size() + ly.size() - lz.size()) / 2);
    d.ka = (uint8_t)(lx.size() - d.k);
    d.kb = (uint8_t)(ly.size() - d.k);
    std::map<int, int> px, py;
    for (size_t i = 0; i < lx.size(); i++) px[lx[i]] = (int)i;
    for (size_t i = 0; i < ly.size(); i++) py[ly[i]] = (int)i;
    // the shared bonds must be the top k bits of both operands, same order
    for (int q = 0; q < d.k; q++)
      if (lx[d.ka + q] != ly[d.kb + q]) return set_error(TNC_ERR_INVALID, "internal: shared bonds misaligned");
    std::vector<int> op(lz.size()), dst(lz.size());
    for (size_t j = 0; j < lz.size(); j++) {
      auto it = px.find(lz[j]);
      if (it != px.end() && it->second < d.ka) {
        op[j] = 0;
        dst[j] = it->second;
      } else {
        auto jt = py.find(lz[j]);
        if (jt == py.end() || jt->second >= d.kb) return set_error(TNC_ERR_INVALID, "internal: output bond not free");
        op[j] = 1;
        dst[j] = jt->second;
      }
    }
    // runs
    int nra = 0, nrb = 0;
    TncRun ra[64], rb[64];
    for (size_t j = 0; j < lz.size();) {
      size_t e = j + 1;
      while (e < lz.size() && op[e] == op[j] && dst[e] == dst[j] + (int)(e - j)) e++;
      TncRun r{(uint8_t)j, (uint8_t)dst[j], (uint8_t)(e - j), 0};
      if (op[j] == 0) ra[nra++] = r;
      else rb[nrb++] = r;
      j = e;
    }
    if (nra <= TNC_MAXRUN && nrb <= TNC_MAXRUN) {
      d.nra = (uint8_t)nra;
      d.nrb = (uint8_t)nrb;
      for (int i = 0; i < nra; i++) d.map.runs.ra[i] = ra[i];
      for (int i = 0; i < nrb; i++) d.map.runs.rb[i] = rb[i];
    } else {
      d.nra = TNC_BITMAP;
      d.nrb = TNC_BITMAP;
      for (size_t j = 0; j < lz.size(); j++) d.map.bit[j] = (uint8_t)((op[j] << 7) | dst[j]);
      low.n_bitmap_steps++;
    }
    low.max_runs = std::max(low.max_runs, std::max(nra, nrb));
  }
  // leaves
  low.leaves.resize(L);
  for (int l = 0; l < L; l++) {
    const Leaf& lf = net.leaves[l];
    LeafDesc& d = low.leaves[l];
    std::memset(&d, 0, sizeof(d));
    d.kind = lf.kind;
    d.rank = (uint8_t)lf.rank();
    if (lf.kind == LK_TABLE) {
      d.table_off = (uint32_t)low.leaf_tables.size();
      const auto& lay = low.layout[l];
      std::vector<int> orig(lay.size());
      for (size_t j = 0; j < lay.size(); j++)
        orig[j] = (int)(std::find(lf.bonds.begin(), lf.bonds.end(), lay[j]) - lf.bonds.begin());
      for (uint32_t o = 0; o < (1u << lf.rank()); o++) {
        uint32_t src = 0;
        for (size_t j = 0; j < lay.size(); j++) src |= ((o >> j) & 1u) << orig[j];
        low.leaf_tables.push_back(lf.table[src]);
      }
    }
  }
  // root permutation: root bit j -> open variable index
  for (int b : low.layout[root]) low.root_perm.push_back((uint8_t)(b - net.first_open_bond));

  std::vector<uint64_t> size(N);
  for (int i = 0; i < N; i++) size[i] = 1ull << tree.nodes[i].bonds.size();
  const int INF = 1 << 30;

  // sequential schedule: internal node z runs at time z - L + 1; leaves exist at 0
  {
    std::vector<int> t0(N), t1(N);
    for (int i = 0; i < N; i++) {
      t0[i] = i < L ? 0 : i - L + 1;
      t1[i] = parent[i] < 0 ? INF : parent[i] - L + 1;
    }
    std::vector<uint64_t> off;
    low.seq_arena_entries = allocate(size, t0, t1, off);
    low.seq_leaf_off.assign(off.begin(), off.begin() + L);
    for (int z = L; z < N; z++) {
      StepDesc d = desc[z];
      d.a_off = off[tree.nodes[z].left];
      d.b_off = off[tree.nodes[z].right];
      d.c_off = off[z];
      low.seq_steps.push_back(d);
    }
    low.seq_root_off = off[root];
  }
  // level schedule
  {
    std::vector<int> lvl(N, 0);
    for (int z = L; z < N; z++) lvl[z] = 1 + std::max(lvl[tree.nodes[z].left], lvl[tree.nodes[z].right]);
    std::vector<int> t0(N), t1(N);
    for (int i = 0; i < N; i++) {
      t0[i] = lvl[i];
      t1[i] = parent[i] < 0 ? INF : lvl[parent[i]];
    }
    std::vector<uint64_t> off;
    low.lvl_arena_entries = allocate(size, t0, t1, off);
    low.lvl_leaf_off.assign(off.begin(), off.begin() + L);
    std::vector<int> ord;
    for (int z = L; z < N; z++) ord.push_back(z);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return lvl[a] < lvl[b]; });
    int nlev = lvl[root];
    low.lvl_start.assign(nlev + 1, 0);
    std::vector<int> idx_of(N, -1);  // node -> index in lvl_steps
    size_t p = 0;
    for (int l = 1; l <= nlev; l++) {
      low.lvl_start[l - 1] = (uint32_t)p;
      uint64_t work = 0;
      while (p < ord.size() && lvl[ord[p]] == l) {
        int z = ord[p];
        StepDesc d = desc[z];
        d.a_off = off[tree.nodes[z].left];
        d.b_off = off[tree.nodes[z].right];
        d.c_off = off[z];
        d.work_lo = (uint32_t)work;
        work += 1ull << d.c;
        idx_of[z] = (int)low.lvl_steps.size();
        low.lvl_steps.push_back(d);
        p++;
      }
    }
    low.lvl_start[nlev] = (uint32_t)p;
    low.lvl_root_off = off[root];
    // producers and consumers among the level schedule's steps
    low.lvl_src_a.assign(low.lvl_steps.size(), -1);
    low.lvl_src_b.assign(low.lvl_steps.size(), -1);
    low.lvl_dst.assign(low.lvl_steps.size(), -1);
    for (int z = L; z < N; z++) {
      const int i = idx_of[z];
      low.lvl_src_a[i] = idx_of[tree.nodes[z].left];
      low.lvl_src_b[i] = idx_of[tree.nodes[z].right];
      if (parent[z] >= 0) low.lvl_dst[i] = idx_of[parent[z]];
    }
    // TNC_PATH_TC_P8: a dense step (unsplit) whose consumer is a dense step
    // reading that operand row-contiguous writes it as fp16 planes, twice the
    // entries' bytes; the same level lifetimes, sizes doubled for those
    const size_t ns = low.lvl_steps.size();
    low.p8_direct.assign(ns, 0);
    std::vector<uint64_t> size8 = size;
    for (int z = L; z < N; z++) {
      const int i = idx_of[z], j = low.lvl_dst[i];
      if (j < 0) continue;
      const StepDesc& d = low.lvl_steps[i];
      const StepDesc& e = low.lvl_steps[j];
      if (!p8_eligible(d) || p8_split_log(d) != 0 || !p8_eligible(e)) continue;
      if (!p8_operand_mn(e, low.lvl_src_a[j] == i ? 0 : 1)) continue;
      low.p8_direct[i] = 1;
      size8[z] = 2 * size[z];
    }
    std::vector<uint64_t> off8;  // 16 entries: fp16 planes start 16-byte aligned (TMA) at 1 residue per entry
    low.p8_arena_entries = allocate(size8, t0, t1, off8, 16);
    low.p8_leaf_off.assign(off8.begin(), off8.begin() + L);
    low.p8_steps = low.lvl_steps;
    for (int z = L; z < N; z++) {
      StepDesc& d = low.p8_steps[idx_of[z]];
      d.a_off = off8[tree.nodes[z].left];
      d.b_off = off8[tree.nodes[z].right];
      d.c_off = off8[z];
    }
    low.p8_root_off = off8[root];
  }
  return TNC_OK;
}

// ---------------------------------------------------------------- validation
//
// Every address a kernel will form from these descriptors, checked on the host:
// each operand/output range lies inside the arena, the output maps cover each
// operand's free bits exactly once, and no output range overlaps a tensor that
// is read or written at the same time (same step, or same level of the level
// schedule).

static bool overlap(uint64_t a, uint64_t na, uint64_t b, uint64_t nb) { return a < b + nb && b < a + na; }

static int check_step(const StepDesc& d, uint64_t arena) {
  const uint64_t nc = 1ull << d.c, na = 1ull << d.a_rank, nb = 1ull << d.b_rank;
  if (d.ka + d.k != d.a_rank || d.kb + d.k != d.b_rank || d.ka + d.kb != d.c)
    return set_error(TNC_ERR_INVALID, "internal: inconsistent step ranks");
  if (d.c_off + nc > arena || d.a_off + na > arena || d.b_off + nb > arena)
    return set_error(TNC_ERR_INVALID, "internal: step range outside the arena");
  if (overlap(d.c_off, nc, d.a_off, na) || overlap(d.c_off, nc, d.b_off, nb))
    return set_error(TNC_ERR_INVALID, "internal: step output overlaps an input");
  uint64_t ca = 0, cb = 0;
  auto add = [](uint64_t& acc, int dst) -> bool {
    if (dst >= 63 || (acc >> dst) & 1ull) return false;
    acc |= 1ull << dst;
    return true;
  };
  if (d.nra == TNC_BITMAP) {
    for (int j = 0; j < d.c; j++) {
      int op = d.map.bit[j] >> 7, dst = d.map.bit[j] & 63;
      if (!add(op ? cb : ca, dst)) return set_error(TNC_ERR_INVALID, "internal: bit map collision");
    }
  } else {
    if (d.nra > TNC_MAXRUN || d.nrb > TNC_MAXRUN) return set_error(TNC_ERR_INVALID, "internal: run count");
    uint64_t covered = 0;
    for (int side = 0; side < 2; side++) {
      const TncRun* rr = side ? d.map.runs.rb : d.map.runs.ra;
      int n = side ? d.nrb : d.nra;
      for (int i = 0; i < n; i++)
        for (int q = 0; q < rr[i].len; q++) {
          int src = rr[i].src + q;
          if (src >= d.c || ((covered >> src) & 1ull)) return set_error(TNC_ERR_INVALID, "internal: run source");
          covered |= 1ull << src;
          if (!add(side ? cb : ca, rr[i].dst + q)) return set_error(TNC_ERR_INVALID, "internal: run collision");
        }
    }
  }
  const uint64_t fa = d.ka >= 64 ? ~0ull : ((1ull << d.ka) - 1), fb = d.kb >= 64 ? ~0ull : ((1ull << d.kb) - 1);
  if (ca != fa || cb != fb) return set_error(TNC_ERR_INVALID, "internal: free bits not covered exactly once");
  return TNC_OK;
}

int validate_lowered(const Network& net, const Tree& tree, Lowered& low) {
  const int L = tree.n_leaves;
  if (tree.nodes.empty()) return TNC_OK;  // empty network: nothing is launched
  if (tree.root < 0 || tree.root >= (int)tree.nodes.size()) return set_error(TNC_ERR_INVALID, "internal: root");
  if ((int)low.leaves.size() != L) return set_error(TNC_ERR_INVALID, "internal: leaf count");
  for (int sched = 0; sched < 2; sched++) {
    const uint64_t arena = sched ? low.lvl_arena_entries : low.seq_arena_entries;
    const auto& leaf_off = sched ? low.lvl_leaf_off : low.seq_leaf_off;
    for (int l = 0; l < L; l++)
      if (leaf_off[l] + (1ull << low.leaves[l].rank) > arena)
        return set_error(TNC_ERR_INVALID, "internal: leaf outside the arena");
    const auto& steps = sched ? low.lvl_steps : low.seq_steps;
    for (const StepDesc& d : steps) {
      int rc = check_step(d, arena);
      if (rc) return rc;
    }
    const uint64_t root_off = sched ? low.lvl_root_off : low.seq_root_off;
    const int root = tree.root;
    const uint64_t root_n = 1ull << tree.nodes[root].bonds.size();
    (void)net;
    if (root_off + root_n > arena) return set_error(TNC_ERR_INVALID, "internal: root outside");
  }
  // level schedule: outputs of a level must not overlap anything the level
  // touches; its 32-bit work offsets (used by the batch kernel) must fit
  bool fits = true;
  for (size_t l = 0; l + 1 < low.lvl_start.size(); l++) {
    uint64_t work = 0;
    for (uint32_t i = low.lvl_start[l]; i < low.lvl_start[l + 1]; i++) work += 1ull << low.lvl_steps[i].c;
    if (work >= (1ull << 32)) fits = false;
  }
  for (size_t l = 0; l + 1 < low.lvl_start.size(); l++) {
    for (uint32_t i = low.lvl_start[l]; i < low.lvl_start[l + 1]; i++) {
      const StepDesc& d = low.lvl_steps[i];
      if (fits) {
        const uint64_t prev_end = i > low.lvl_start[l] ? (uint64_t)low.lvl_steps[i - 1].work_lo +
                                                             (1ull << low.lvl_steps[i - 1].c)
                                                       : 0;
        if ((uint64_t)d.work_lo != prev_end) return set_error(TNC_ERR_INVALID, "internal: work offsets");
      }
      for (uint32_t j = low.lvl_start[l]; j < low.lvl_start[l + 1]; j++) {
        if (i == j) continue;
        const StepDesc& e = low.lvl_steps[j];
        const uint64_t nc = 1ull << d.c;
        if (overlap(d.c_off, nc, e.c_off, 1ull << e.c) || overlap(d.c_off, nc, e.a_off, 1ull << e.a_rank) ||
            overlap(d.c_off, nc, e.b_off, 1ull << e.b_rank))
          return set_error(TNC_ERR_INVALID, "internal: level outputs overlap");
      }
    }
  }
  {  // the TNC_PATH_TC_P8 layout: direct outputs take twice their entries
    const size_t ns = low.lvl_steps.size();
    if (low.p8_steps.size() != ns || low.p8_direct.size() != ns || low.p8_leaf_off.size() != (size_t)L)
      return set_error(TNC_ERR_INVALID, "internal: p8 layout size");
    const uint64_t arena = low.p8_arena_entries;
    for (int l = 0; l < L; l++)
      if (low.p8_leaf_off[l] + (1ull << low.leaves[l].rank) > arena)
        return set_error(TNC_ERR_INVALID, "internal: leaf outside the p8 arena");
    auto ext = [&](int i, int rank) -> uint64_t { return (1ull << rank) * (i >= 0 && low.p8_direct[i] ? 2 : 1); };
    std::vector<uint64_t> nc(ns), na(ns), nb(ns);
    for (size_t i = 0; i < ns; i++) {
      const StepDesc& d = low.p8_steps[i];
      int rc = check_step(d, arena);
      if (rc) return rc;
      nc[i] = ext((int)i, d.c);
      na[i] = ext(low.lvl_src_a[i], d.a_rank);
      nb[i] = ext(low.lvl_src_b[i], d.b_rank);
      if (d.c_off + nc[i] > arena || d.a_off + na[i] > arena || d.b_off + nb[i] > arena)
        return set_error(TNC_ERR_INVALID, "internal: fp16 planes outside the p8 arena");
      if (overlap(d.c_off, nc[i], d.a_off, na[i]) || overlap(d.c_off, nc[i], d.b_off, nb[i]))
        return set_error(TNC_ERR_INVALID, "internal: p8 output overlaps an input");
      if (low.p8_direct[i] && (low.lvl_dst[i] < 0 || p8_split_log(d) != 0))
        return set_error(TNC_ERR_INVALID, "internal: direct planes without a dense consumer");
    }
    for (size_t l = 0; l + 1 < low.lvl_start.size(); l++)
      for (uint32_t i = low.lvl_start[l]; i < low.lvl_start[l + 1]; i++)
        for (uint32_t j = low.lvl_start[l]; j < low.lvl_start[l + 1]; j++) {
          if (i == j) continue;
          const StepDesc& d = low.p8_steps[i];
          const StepDesc& e = low.p8_steps[j];
          if (overlap(d.c_off, nc[i], e.c_off, nc[j]) || overlap(d.c_off, nc[i], e.a_off, na[j]) ||
              overlap(d.c_off, nc[i], e.b_off, nb[j]))
            return set_error(TNC_ERR_INVALID, "internal: p8 level outputs overlap");
        }
    if (low.p8_root_off + (1ull << tree.nodes[tree.root].bonds.size()) > arena)
      return set_error(TNC_ERR_INVALID, "internal: root outside the p8 arena");
  }
  if (!fits) return TNC_OK;  // lvl_fits stays false: the batch kernel refuses this plan
  low.lvl_fits = true;
  return TNC_OK;
}

}  // namespace tnc

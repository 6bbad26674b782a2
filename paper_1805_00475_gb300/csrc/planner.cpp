// Host planner: contraction trees from the paper's ordering heuristics
// (Sec. 3.1.1) and their exact cost (Sec. 2.2, Corollary 2, Sec. 4 "lazy").
//
//   tensor-greedy : repeatedly contract the connected pair whose result has the
//                   smallest rank.
//   tensor-METIS  : recursive balanced min-cut bisection down to single
//                   tensors, each split the better of `tries` randomised runs;
//                   the separator hierarchy is the contraction tree (smallest,
//                   i.e. deepest, separators contracted first).  METIS itself
//                   is replaced by an own multilevel bisection (heavy-edge
//                   matching, greedy graph growing, Fiduccia-Mattheyses).
//   tensor-GN     : Girvan-Newman; delete the edge of highest betweenness until
//                   a community splits; the dendrogram is the contraction tree.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <queue>
#include <set>

#include "tnc_internal.h"

namespace tnc {

// --------------------------------------------------------------- tree basics

static std::vector<int> sym_diff(const std::vector<int>& a, const std::vector<int>& b) {
  std::vector<int> out;
  out.reserve(a.size() + b.size());
  std::set_symmetric_difference(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(out));
  return out;
}

static int shared_count(const std::vector<int>& a, const std::vector<int>& b) {
  int k = 0;
  size_t i = 0, j = 0;
  while (i < a.size() && j < b.size()) {
    if (a[i] < b[j]) i++;
    else if (a[i] > b[j]) j++;
    else { k++; i++; j++; }
  }
  return k;
}

static void init_leaves(const Network& net, Tree& t) {
  t.nodes.clear();
  t.n_leaves = net.n_leaves();
  t.nodes.resize(net.n_leaves());
  for (int i = 0; i < net.n_leaves(); i++) {
    t.nodes[i].bonds = net.leaves[i].bonds;
    std::sort(t.nodes[i].bonds.begin(), t.nodes[i].bonds.end());
  }
  t.root = net.n_leaves() == 1 ? 0 : -1;
}

static int merge(Tree& t, int a, int b) {
  Node n;
  n.left = a;
  n.right = b;
  n.bonds = sym_diff(t.nodes[a].bonds, t.nodes[b].bonds);
  t.nodes.push_back(std::move(n));
  int id = (int)t.nodes.size() - 1;
  t.root = id;
  return id;
}

TreeCost tree_cost(const Tree& t) {
  TreeCost c;
  std::vector<int> depth(t.nodes.size(), 0);
  for (int i = 0; i < t.n_leaves; i++) c.max_rank = std::max(c.max_rank, (int)t.nodes[i].bonds.size());
  for (size_t i = t.n_leaves; i < t.nodes.size(); i++) {
    const Node& n = t.nodes[i];
    const int a = (int)t.nodes[n.left].bonds.size(), b = (int)t.nodes[n.right].bonds.size();
    const int k = shared_count(t.nodes[n.left].bonds, t.nodes[n.right].bonds);
    const int r = (int)n.bonds.size();
    c.max_rank = std::max(c.max_rank, r);
    c.macs += std::ldexp(1.0, a + b - k);
    c.entries += std::ldexp(1.0, a) + std::ldexp(1.0, b) + std::ldexp(1.0, r);
    depth[i] = 1 + std::max(depth[n.left], depth[n.right]);
    c.depth = std::max(c.depth, depth[i]);
  }
  return c;
}

// Merge every remaining live subtree root into one tree: connected pairs are
// impossible here (callers finish components first), so these are scalar or
// open-bond outer products; smallest rank first, ties by id.
static void finish_outer(Tree& t, std::vector<int> live) {
  while (live.size() > 1) {
    std::sort(live.begin(), live.end(), [&](int x, int y) {
      size_t rx = t.nodes[x].bonds.size(), ry = t.nodes[y].bonds.size();
      return rx != ry ? rx < ry : x < y;
    });
    int a = live[0], b = live[1];
    int c = merge(t, std::min(a, b), std::max(a, b));
    live.erase(live.begin(), live.begin() + 2);
    live.push_back(c);
  }
  if (live.size() == 1) t.root = live[0];
}

// ------------------------------------------------------------ tensor-greedy

// Adjacency of live subtree roots: node -> (neighbour -> shared bond count).
struct Adjacency {
  std::vector<std::map<int, int>> nb;
};

static void greedy_from(const Network& net, Tree& t, std::vector<char>& live) {
  (void)net;
  Adjacency adj;
  adj.nb.resize(t.nodes.size() * 2 + 2);
  std::map<int, std::vector<int>> owners;  // bond -> live owners
  for (size_t i = 0; i < t.nodes.size(); i++)
    if (live[i])
      for (int b : t.nodes[i].bonds) owners[b].push_back((int)i);
  for (auto& kv : owners)
    if (kv.second.size() == 2) {
      adj.nb[kv.second[0]][kv.second[1]]++;
      adj.nb[kv.second[1]][kv.second[0]]++;
    }
  for (;;) {
    int ba = -1, bb = -1;
    long br = 0, bm = 0;
    for (size_t i = 0; i < t.nodes.size(); i++) {
      if (!live[i]) continue;
      for (auto& kv : adj.nb[i]) {
        int j = kv.first;
        if (j <= (int)i || !live[j]) continue;
        long a = (long)t.nodes[i].bonds.size(), b = (long)t.nodes[j].bonds.size(), k = kv.second;
        long r = a + b - 2 * k, mac = a + b - k;
        bool better = ba < 0 || r < br || (r == br && (mac < bm || (mac == bm && ((int)i < ba || ((int)i == ba && j < bb)))));
        if (better) {
          ba = (int)i;
          bb = j;
          br = r;
          bm = mac;
        }
      }
    }
    if (ba < 0) break;
    int c = merge(t, ba, bb);
    if ((size_t)c >= live.size()) live.resize(c + 1, 0);
    if ((size_t)c >= adj.nb.size()) adj.nb.resize(c + 1);
    live[ba] = live[bb] = 0;
    live[c] = 1;
    std::map<int, int> nc;
    for (int src : {ba, bb})
      for (auto& kv : adj.nb[src])
        if (kv.first != ba && kv.first != bb) nc[kv.first] += kv.second;
    for (auto& kv : nc) {
      auto& m = adj.nb[kv.first];
      m.erase(ba);
      m.erase(bb);
      m[c] = kv.second;
    }
    adj.nb[c] = nc;
    adj.nb[ba].clear();
    adj.nb[bb].clear();
  }
  std::vector<int> rest;
  for (size_t i = 0; i < t.nodes.size(); i++)
    if (i < live.size() && live[i]) rest.push_back((int)i);
  finish_outer(t, rest);
}

int plan_greedy(const Network& net, Tree& t) {
  init_leaves(net, t);
  std::vector<char> live(t.nodes.size(), 1);
  greedy_from(net, t, live);
  return TNC_OK;
}

void tree_from_merges(const Network& net, const std::vector<std::pair<int, int>>& merges, Tree& t) {
  init_leaves(net, t);
  std::vector<char> live(t.nodes.size(), 1);
  for (auto& p : merges) {
    int c = merge(t, p.first, p.second);
    live.resize(c + 1, 0);
    live[p.first] = live[p.second] = 0;
    live[c] = 1;
  }
  greedy_from(net, t, live);
}

// ------------------------------------------------------- weighted graphs

struct WGraph {
  int n = 0;
  std::vector<int> xadj, adj, ew, vw;  // CSR; ew = edge weight; vw = vertex weight
  int total_vw() const { return std::accumulate(vw.begin(), vw.end(), 0); }
};

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
  int below(int n) { return (int)(next() % (uint64_t)n); }
};

// Induced subgraph of the network's leaf graph on `verts` (edge weight = number
// of bonds between two leaves).
static WGraph induced(const Network& net, const std::vector<int>& verts) {
  WGraph g;
  g.n = (int)verts.size();
  std::map<int, int> loc;
  for (int i = 0; i < g.n; i++) loc[verts[i]] = i;
  std::vector<std::map<int, int>> nb(g.n);
  for (int i = 0; i < g.n; i++) {
    for (int b : net.leaves[verts[i]].bonds) {
      int e0 = net.bond_end0[b], e1 = net.bond_end1[b];
      int other = e0 == verts[i] ? e1 : e0;
      if (other < 0) continue;
      auto it = loc.find(other);
      if (it == loc.end() || it->second == i) continue;
      nb[i][it->second]++;
    }
  }
  g.xadj.assign(g.n + 1, 0);
  for (int i = 0; i < g.n; i++) {
    g.xadj[i + 1] = g.xadj[i] + (int)nb[i].size();
    for (auto& kv : nb[i]) {
      g.adj.push_back(kv.first);
      g.ew.push_back(kv.second);
    }
  }
  g.vw.assign(g.n, 1);
  return g;
}

static long cut_of(const WGraph& g, const std::vector<uint8_t>& side) {
  long c = 0;
  for (int u = 0; u < g.n; u++)
    for (int e = g.xadj[u]; e < g.xadj[u + 1]; e++)
      if (side[u] != side[g.adj[e]]) c += g.ew[e];
  return c / 2;
}

static int max_part(int total) { return std::max((total + 1) / 2, (int)std::floor(0.515 * total)); }

// Fiduccia-Mattheyses refinement under the balance bound.
static void fm_refine(const WGraph& g, std::vector<uint8_t>& side, int passes) {
  const int W = g.total_vw(), cap = max_part(W);
  for (int pass = 0; pass < passes; pass++) {
    std::vector<long> gain(g.n, 0);
    int pw[2] = {0, 0};
    for (int u = 0; u < g.n; u++) {
      pw[side[u]] += g.vw[u];
      for (int e = g.xadj[u]; e < g.xadj[u + 1]; e++)
        gain[u] += side[g.adj[e]] != side[u] ? g.ew[e] : -g.ew[e];
    }
    std::vector<char> locked(g.n, 0);
    std::vector<int> moves;
    long cur = 0, best = 0;
    size_t best_len = 0;
    for (int step = 0; step < g.n; step++) {
      int bu = -1;
      for (int u = 0; u < g.n; u++) {
        if (locked[u]) continue;
        int to = 1 - side[u];
        if (pw[to] + g.vw[u] > cap) continue;
        if (bu < 0 || gain[u] > gain[bu]) bu = u;
      }
      if (bu < 0) break;
      int from = side[bu], to = 1 - from;
      cur -= gain[bu];
      side[bu] = (uint8_t)to;
      pw[from] -= g.vw[bu];
      pw[to] += g.vw[bu];
      locked[bu] = 1;
      moves.push_back(bu);
      gain[bu] = -gain[bu];
      for (int e = g.xadj[bu]; e < g.xadj[bu + 1]; e++) {
        int v = g.adj[e];
        gain[v] += side[v] == to ? -2 * g.ew[e] : 2 * g.ew[e];
      }
      if (cur < best) {
        best = cur;
        best_len = moves.size();
      }
    }
    for (size_t i = moves.size(); i > best_len; i--) side[moves[i - 1]] ^= 1;
    if (best_len == 0) break;
  }
}

// Greedy graph growing from a random start vertex (Sec. 3.1.1: METIS starts
// from a randomly chosen vertex).
static std::vector<uint8_t> grow(const WGraph& g, Rng& rng) {
  std::vector<uint8_t> side(g.n, 0);
  const int W = g.total_vw();
  int w1 = 0;
  std::vector<long> conn(g.n, 0);
  std::vector<char> in(g.n, 0);
  int start = rng.below(g.n);
  while (2 * w1 < W) {
    int pick = -1;
    if (w1 == 0) pick = start;
    else {
      for (int u = 0; u < g.n; u++) {
        if (in[u] || conn[u] <= 0) continue;
        if (pick < 0 || conn[u] > conn[pick]) pick = u;
      }
      if (pick < 0) {  // disconnected: any unassigned vertex
        std::vector<int> rest;
        for (int u = 0; u < g.n; u++)
          if (!in[u]) rest.push_back(u);
        if (rest.empty()) break;
        pick = rest[rng.below((int)rest.size())];
      }
    }
    if (w1 > 0 && 2 * (w1 + g.vw[pick]) > W + g.vw[pick]) break;
    in[pick] = 1;
    side[pick] = 1;
    w1 += g.vw[pick];
    for (int e = g.xadj[pick]; e < g.xadj[pick + 1]; e++) conn[g.adj[e]] += g.ew[e];
  }
  return side;
}

// Heavy-edge matching coarsening step; returns coarse graph and the map.
static WGraph coarsen(const WGraph& g, Rng& rng, std::vector<int>& cmap) {
  std::vector<int> ord(g.n);
  std::iota(ord.begin(), ord.end(), 0);
  for (int i = g.n - 1; i > 0; i--) std::swap(ord[i], ord[rng.below(i + 1)]);
  std::vector<int> match(g.n, -1);
  for (int u : ord) {
    if (match[u] >= 0) continue;
    int best = -1, bw = -1;
    for (int e = g.xadj[u]; e < g.xadj[u + 1]; e++) {
      int v = g.adj[e];
      if (match[v] >= 0 || v == u) continue;
      if (g.ew[e] > bw) {
        bw = g.ew[e];
        best = v;
      }
    }
    if (best >= 0) {
      match[u] = best;
      match[best] = u;
    } else match[u] = u;
  }
  cmap.assign(g.n, -1);
  int nc = 0;
  for (int u = 0; u < g.n; u++) {
    if (cmap[u] >= 0) continue;
    cmap[u] = nc;
    if (match[u] != u) cmap[match[u]] = nc;
    nc++;
  }
  WGraph c;
  c.n = nc;
  c.vw.assign(nc, 0);
  std::vector<std::map<int, int>> nb(nc);
  for (int u = 0; u < g.n; u++) {
    c.vw[cmap[u]] += g.vw[u];
    for (int e = g.xadj[u]; e < g.xadj[u + 1]; e++) {
      int cu = cmap[u], cv = cmap[g.adj[e]];
      if (cu != cv) nb[cu][cv] += g.ew[e];
    }
  }
  c.xadj.assign(nc + 1, 0);
  for (int i = 0; i < nc; i++) {
    c.xadj[i + 1] = c.xadj[i] + (int)nb[i].size();
    for (auto& kv : nb[i]) {
      c.adj.push_back(kv.first);
      c.ew.push_back(kv.second);
    }
  }
  return c;
}

// One multilevel bisection run.
static std::vector<uint8_t> bisect_once(const WGraph& g0, Rng& rng) {
  std::vector<WGraph> levels{g0};
  std::vector<std::vector<int>> maps;
  while (levels.back().n > 24) {
    std::vector<int> cm;
    WGraph c = coarsen(levels.back(), rng, cm);
    if (c.n > (int)(0.9 * levels.back().n)) break;
    maps.push_back(cm);
    levels.push_back(std::move(c));
  }
  const WGraph& gc = levels.back();
  std::vector<uint8_t> best;
  long bc = -1;
  for (int a = 0; a < 4; a++) {
    std::vector<uint8_t> s = grow(gc, rng);
    fm_refine(gc, s, 8);
    long c = cut_of(gc, s);
    if (bc < 0 || c < bc) {
      bc = c;
      best = s;
    }
  }
  std::vector<uint8_t> side = best;
  for (int l = (int)levels.size() - 2; l >= 0; l--) {
    std::vector<uint8_t> fine(levels[l].n);
    for (int u = 0; u < levels[l].n; u++) fine[u] = side[maps[l][u]];
    side.swap(fine);
    fm_refine(levels[l], side, 8);
  }
  return side;
}

// Recursive bisection of `verts` (leaf ids) into a subtree; returns its node.
static int bisect_rec(const Network& net, Tree& t, const std::vector<int>& verts, int tries, Rng& rng) {
  if (verts.size() == 1) return verts[0];
  if (verts.size() == 2) return merge(t, std::min(verts[0], verts[1]), std::max(verts[0], verts[1]));
  WGraph g = induced(net, verts);
  std::vector<uint8_t> best;
  long bc = -1;
  for (int k = 0; k < tries; k++) {
    std::vector<uint8_t> s = bisect_once(g, rng);
    long c = cut_of(g, s);
    if (bc < 0 || c < bc) {
      bc = c;
      best = s;
    }
  }
  std::vector<int> p0, p1;
  for (size_t i = 0; i < verts.size(); i++) (best[i] ? p1 : p0).push_back(verts[i]);
  if (p0.empty() || p1.empty()) {  // degenerate split: halve by index
    p0.assign(verts.begin(), verts.begin() + verts.size() / 2);
    p1.assign(verts.begin() + verts.size() / 2, verts.end());
  }
  int l = bisect_rec(net, t, p0, tries, rng);
  int r = bisect_rec(net, t, p1, tries, rng);
  return merge(t, l, r);
}

int plan_bisect(const Network& net, int tries, uint64_t seed, Tree& t) {
  init_leaves(net, t);
  if (net.n_leaves() <= 1) return TNC_OK;
  Rng rng(seed ^ 0x5DEECE66Dull);
  std::vector<int> all(net.n_leaves());
  std::iota(all.begin(), all.end(), 0);
  t.root = bisect_rec(net, t, all, std::max(1, tries), rng);
  return TNC_OK;
}

// ------------------------------------------------------------ tensor-GN

// Simple graph (parallel bonds merged) of the leaves with alive flags.
struct GNGraph {
  int n = 0;
  std::vector<std::vector<std::pair<int, int>>> nb;  // (neighbour, edge id)
  std::vector<int> eu, ev;
  std::vector<char> alive;
};

// Buffers of the betweenness computation, reused across a whole GN run.
struct GNScratch {
  std::vector<int> loc;               // leaf -> index in the current vertex set
  std::vector<int> off, adj_v, adj_e; // alive edges inside the set, per vertex (g.nb order)
  std::vector<int> dist, order;
  std::vector<double> sigma, delta;
};

// Edge betweenness (Brandes 2001, unweighted) restricted to vertex set `vs`.
// The alive edges inside `vs` are first gathered into per-vertex lists that
// keep g.nb's neighbour order, so the |vs| breadth-first searches touch only
// them; sources, visits and sums run in the same order as a search over g.nb
// itself, so every sum is formed in the same order.
static void betweenness(const GNGraph& g, const std::vector<int>& vs, const std::vector<char>& inset,
                        std::vector<double>& eb, GNScratch& w) {
  std::fill(eb.begin(), eb.end(), 0.0);
  const int n = (int)vs.size();
  w.loc.resize(g.n);
  for (int i = 0; i < n; i++) w.loc[vs[i]] = i;
  w.off.assign(n + 1, 0);
  w.adj_v.clear();
  w.adj_e.clear();
  for (int i = 0; i < n; i++) {
    for (auto& pe : g.nb[vs[i]]) {
      if (!g.alive[pe.second] || !inset[pe.first]) continue;
      w.adj_v.push_back(w.loc[pe.first]);
      w.adj_e.push_back(pe.second);
    }
    w.off[i + 1] = (int)w.adj_v.size();
  }
  w.dist.assign(n, -1);
  w.sigma.assign(n, 0.0);
  w.delta.assign(n, 0.0);
  w.order.resize(n);
  int* dist = w.dist.data();
  double* sigma = w.sigma.data();
  double* delta = w.delta.data();
  int* order = w.order.data();
  const int* off = w.off.data();
  const int* av = w.adj_v.data();
  const int* ae = w.adj_e.data();
  for (int s = 0; s < n; s++) {
    for (int v = 0; v < n; v++) {
      dist[v] = -1;
      sigma[v] = 0;
      delta[v] = 0;
    }
    dist[s] = 0;
    sigma[s] = 1;
    order[0] = s;
    int head = 0, tail = 1;  // order[] is the queue and the visit order
    while (head < tail) {
      const int u = order[head++];
      for (int j = off[u]; j < off[u + 1]; j++) {
        const int v = av[j];
        if (dist[v] < 0) {
          dist[v] = dist[u] + 1;
          order[tail++] = v;
        }
        if (dist[v] == dist[u] + 1) sigma[v] += sigma[u];
      }
    }
    for (int i = tail; i-- > 0;) {
      const int x = order[i];
      for (int j = off[x]; j < off[x + 1]; j++) {
        const int v = av[j];
        if (dist[v] == dist[x] - 1) {
          const double c = sigma[v] / sigma[x] * (1.0 + delta[x]);
          eb[ae[j]] += c;
          delta[v] += c;
        }
      }
    }
  }
}

static std::vector<std::vector<int>> components(const GNGraph& g, const std::vector<int>& vs,
                                                const std::vector<char>& inset) {
  std::vector<std::vector<int>> comps;
  std::vector<char> seen(g.n, 0);
  for (int s : vs) {
    if (seen[s]) continue;
    std::vector<int> comp{s};
    seen[s] = 1;
    for (size_t h = 0; h < comp.size(); h++) {
      int u = comp[h];
      for (auto& pe : g.nb[u]) {
        int v = pe.first;
        if (!g.alive[pe.second] || !inset[v] || seen[v]) continue;
        seen[v] = 1;
        comp.push_back(v);
      }
    }
    std::sort(comp.begin(), comp.end());
    comps.push_back(comp);
  }
  return comps;
}

static int gn_rec(Tree& t, GNGraph& g, std::vector<int> vs, GNScratch& w) {
  if (vs.size() == 1) return vs[0];
  std::vector<char> inset(g.n, 0);
  for (int v : vs) inset[v] = 1;
  std::vector<double> eb(g.eu.size(), 0.0);
  for (;;) {
    auto comps = components(g, vs, inset);
    if (comps.size() > 1) {
      std::vector<int> roots;
      for (auto& c : comps) roots.push_back(gn_rec(t, g, c, w));
      // combine the communities smallest rank first (a binary dendrogram)
      while (roots.size() > 1) {
        std::sort(roots.begin(), roots.end(), [&](int x, int y) {
          size_t rx = t.nodes[x].bonds.size(), ry = t.nodes[y].bonds.size();
          return rx != ry ? rx < ry : x < y;
        });
        int c = merge(t, roots[0], roots[1]);
        roots.erase(roots.begin(), roots.begin() + 2);
        roots.push_back(c);
      }
      return roots[0];
    }
    betweenness(g, vs, inset, eb, w);
    int best = -1;
    for (size_t e = 0; e < g.eu.size(); e++) {
      if (!g.alive[e] || !inset[g.eu[e]] || !inset[g.ev[e]]) continue;
      if (best < 0 || eb[e] > eb[best] + 1e-9) best = (int)e;
    }
    if (best < 0) break;  // no edges left (cannot happen for |vs| > 1 connected)
    g.alive[best] = 0;
  }
  return vs[0];
}

int plan_gn(const Network& net, Tree& t) {
  init_leaves(net, t);
  if (net.n_leaves() <= 1) return TNC_OK;
  GNGraph g;
  g.n = net.n_leaves();
  g.nb.resize(g.n);
  std::set<std::pair<int, int>> seen;
  for (int b = 0; b < net.n_bonds; b++) {
    int u = net.bond_end0[b], v = net.bond_end1[b];
    if (u < 0 || v < 0 || u == v) continue;
    auto key = std::make_pair(std::min(u, v), std::max(u, v));
    if (seen.count(key)) continue;
    seen.insert(key);
  }
  for (auto& kv : seen) {  // edge ids in (u, v) order
    int id = (int)g.eu.size();
    g.eu.push_back(kv.first);
    g.ev.push_back(kv.second);
    g.nb[kv.first].push_back({kv.second, id});
    g.nb[kv.second].push_back({kv.first, id});
  }
  g.alive.assign(g.eu.size(), 1);
  std::vector<int> all(g.n);
  std::iota(all.begin(), all.end(), 0);
  GNScratch w;
  t.root = gn_rec(t, g, all, w);
  return TNC_OK;
}

// ------------------------------------------------------------ dispatcher

int plan_tree(const Network& net, const tnc_plan_opts& o, Tree& t) {
  switch (o.heuristic) {
    case TNC_PLAN_GREEDY: return plan_greedy(net, t);
    case TNC_PLAN_BISECT: return plan_bisect(net, o.tries > 0 ? o.tries : 2, o.seed, t);
    case TNC_PLAN_GN: return plan_gn(net, t);
    case TNC_PLAN_EXPLICIT: {
      if (o.n_order < 0 || (o.n_order > 0 && !o.order)) return set_error(TNC_ERR_INVALID, "bad explicit order");
      std::vector<std::pair<int, int>> m;
      std::vector<char> live(net.n_leaves() + o.n_order + 1, 0);
      for (int i = 0; i < net.n_leaves(); i++) live[i] = 1;
      for (int i = 0; i < o.n_order; i++) {
        int a = o.order[2 * i], b = o.order[2 * i + 1];
        int top = net.n_leaves() + i;
        if (a < 0 || b < 0 || a >= top || b >= top || a == b || !live[a] || !live[b])
          return set_error(TNC_ERR_INVALID, "explicit order names a dead or unknown tensor");
        live[a] = live[b] = 0;
        live[top] = 1;
        m.push_back({a, b});
      }
      tree_from_merges(net, m, t);
      return TNC_OK;
    }
    case TNC_PLAN_BEST: {
      Tree cand[3];
      plan_greedy(net, cand[0]);
      plan_bisect(net, o.tries > 0 ? o.tries : 2, o.seed, cand[1]);
      plan_gn(net, cand[2]);
      int best = 0;
      TreeCost bc = tree_cost(cand[0]);
      for (int i = 1; i < 3; i++) {
        TreeCost c = tree_cost(cand[i]);
        if (c.max_rank < bc.max_rank || (c.max_rank == bc.max_rank && c.macs < bc.macs)) {
          bc = c;
          best = i;
        }
      }
      t = std::move(cand[best]);
      return TNC_OK;
    }
    case TNC_PLAN_PORTFOLIO: {
      // tensor-greedy, tensor-GN and 8 independently seeded tensor-METIS
      // runs; the cheapest exact cost (max rank, then MACs) is kept
      plan_greedy(net, t);
      TreeCost bc = tree_cost(t);
      for (int i = 0; i < 9; i++) {
        Tree c;
        if (i == 0) plan_gn(net, c);
        else plan_bisect(net, o.tries > 0 ? o.tries : 2, o.seed + 0x9E3779B97F4A7C15ull * (uint64_t)i, c);
        const TreeCost cc = tree_cost(c);
        if (cc.max_rank < bc.max_rank || (cc.max_rank == bc.max_rank && cc.macs < bc.macs)) {
          bc = cc;
          t = std::move(c);
        }
      }
      return TNC_OK;
    }
    case TNC_PLAN_COARSEN: return plan_coarsen(net, o, t);
  }
  return set_error(TNC_ERR_INVALID, "unknown heuristic");
}

}  // namespace tnc

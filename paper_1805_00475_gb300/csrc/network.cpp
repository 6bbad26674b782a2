// Formula -> tensor network (Sec. 2.1), certified count bound, primes, errors.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>

#include "tnc_internal.h"

namespace tnc {

static thread_local std::string g_err;

int set_error(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
void clear_error() { g_err.clear(); }
const char* last_error_cstr() { return g_err.c_str(); }

// ---------------------------------------------------------------- primes

static uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t m) {
  return (uint64_t)((unsigned __int128)a * b % m);
}
static uint64_t powmod64(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  a %= m;
  while (e) {
    if (e & 1) r = mulmod64(r, a, m);
    a = mulmod64(a, a, m);
    e >>= 1;
  }
  return r;
}

// Deterministic Miller-Rabin: bases {2,3,5,7} decide primality for every
// n < 3,215,031,751 (Jaeschke 1993), which covers all of u32 below 2^31.
bool is_prime_u32(uint32_t n) {
  if (n < 2) return false;
  for (uint32_t p : {2u, 3u, 5u, 7u}) {
    if (n == p) return true;
    if (n % p == 0) return false;
  }
  uint64_t d = n - 1;
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    s++;
  }
  for (uint64_t a : {2ull, 3ull, 5ull, 7ull}) {
    uint64_t x = powmod64(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; r++) {
      x = mulmod64(x, x, n);
      if (x == n - 1) {
        comp = false;
        break;
      }
    }
    if (comp) return false;
  }
  return true;
}

std::vector<uint32_t> default_primes(int n) {
  std::vector<uint32_t> out;
  for (uint32_t x = kDefaultPrimeBound - 1; (int)out.size() < n && x > 2; x -= 2)
    if (is_prime_u32(x)) out.push_back(x);
  return out;
}

std::vector<uint32_t> default_primes_p8(int n) {
  std::vector<uint32_t> out;
  for (uint32_t x = kP8PrimeMax; (int)out.size() < n && x > 2; x -= 2)
    if (is_prime_u32(x)) out.push_back(x);
  return out;
}

// ---------------------------------------------------------------- network

static int find_root(std::vector<int>& p, int x) {
  while (p[x] != x) {
    p[x] = p[p[x]];
    x = p[x];
  }
  return x;
}

// Weight mass of a clause tensor: the sum of its entries.
static double clause_mass(const Leaf& l) {
  const int d = l.rank();
  switch (l.kind) {
    case LK_1IN3: return (double)d;
    case LK_OR:
    case LK_NAND: return std::ldexp(1.0, d) - 1.0;
    case LK_TABLE: {
      double s = 0;
      for (uint32_t v : l.table) s += (double)v;
      return s;
    }
  }
  return std::ldexp(1.0, d);
}

int build_network(const tnc_formula* f, Network& net) {
  if (!f) return set_error(TNC_ERR_INVALID, "formula is NULL");
  if (f->n_vars < 0 || f->n_cons < 0) return set_error(TNC_ERR_INVALID, "negative sizes");
  if (f->n_cons > 0 && (!f->arity || !f->kind)) return set_error(TNC_ERR_INVALID, "arity/kind NULL");
  if (f->n_open < 0 || f->n_open > 20) return set_error(TNC_ERR_INVALID, "n_open must be in [0, 20]");
  if (f->n_open > 0 && !f->open_vars) return set_error(TNC_ERR_INVALID, "open_vars NULL");
  net = Network();
  net.n_vars = f->n_vars;
  net.n_cons = f->n_cons;
  const int m = f->n_cons, n = f->n_vars;
  long total_occ = 0;
  for (int c = 0; c < m; c++) {
    if (f->arity[c] < 0 || f->arity[c] > 20) return set_error(TNC_ERR_INVALID, "clause arity must be in [0, 20]");
    if (f->kind[c] > TNC_TABLE) return set_error(TNC_ERR_INVALID, "unknown clause kind");
    if (f->kind[c] == TNC_TABLE && !f->table) return set_error(TNC_ERR_INVALID, "TABLE clause without table");
    total_occ += f->arity[c];
  }
  if (total_occ > 0 && !f->var_of) return set_error(TNC_ERR_INVALID, "var_of NULL");
  std::vector<int> is_open(n, -1);
  for (int i = 0; i < f->n_open; i++) {
    int v = f->open_vars[i];
    if (v < 0 || v >= n || is_open[v] >= 0) return set_error(TNC_ERR_INVALID, "bad or repeated open variable");
    is_open[v] = i;
    net.open_vars.push_back(v);
  }
  net.leaves.resize((size_t)m + (size_t)n);
  net.n_bonds = (int)total_occ + f->n_open;
  net.first_open_bond = (int)total_occ;
  net.bond_end0.assign(net.n_bonds, -1);
  net.bond_end1.assign(net.n_bonds, -1);
  long s = 0, toff = 0;
  for (int c = 0; c < m; c++) {
    Leaf& L = net.leaves[c];
    L.kind = f->kind[c];
    const int d = f->arity[c];
    for (int j = 0; j < d; j++) {
      int v = f->var_of[s + j];
      if (v < 0 || v >= n) return set_error(TNC_ERR_INVALID, "variable index out of range");
      int b = (int)(s + j);
      L.bonds.push_back(b);
      net.leaves[m + v].bonds.push_back(b);
      net.bond_end0[b] = c;
      net.bond_end1[b] = m + v;
    }
    if (L.kind == LK_TABLE) {
      L.table.assign(f->table + toff, f->table + toff + (1L << d));
      toff += 1L << d;
    }
    s += d;
  }
  for (int v = 0; v < n; v++) {
    Leaf& L = net.leaves[m + v];
    L.kind = LK_COPY;
    if (is_open[v] >= 0) {
      int b = net.first_open_bond + is_open[v];
      L.bonds.push_back(b);
      net.bond_end0[b] = m + v;
    }
    if (L.rank() > 32) return set_error(TNC_ERR_TOO_LARGE, "a variable occurs in more than 32 clauses");
  }
  // connected components (union-find over bonds)
  std::vector<int> par(net.leaves.size());
  std::iota(par.begin(), par.end(), 0);
  for (int b = 0; b < net.n_bonds; b++) {
    if (net.bond_end1[b] < 0) continue;
    int x = find_root(par, net.bond_end0[b]), y = find_root(par, net.bond_end1[b]);
    if (x != y) par[x] = y;
  }
  int comps = 0;
  for (size_t i = 0; i < par.size(); i++)
    if (find_root(par, (int)i) == (int)i) comps++;
  net.n_components = comps;

  // Certified upper bound on every count entry: pick variable-disjoint clauses
  // greedily; each such clause c allows at most mass(c) weighted assignments
  // of its d variables, and every other variable contributes at most 2; every
  // remaining clause contributes at most its largest entry.
  std::vector<char> used(n, 0), picked(m, 0);
  std::vector<int> ord(m);
  std::iota(ord.begin(), ord.end(), 0);
  auto gain = [&](int c) {
    const Leaf& L = net.leaves[c];
    double mass = clause_mass(L);
    return (double)L.rank() - (mass > 0 ? std::log2(mass) : -1e300);
  };
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return gain(a) > gain(b); });
  double lb = 0.0;
  int free_vars = n;
  s = 0;
  std::vector<long> voff(m + 1, 0);
  for (int c = 0; c < m; c++) voff[c + 1] = voff[c] + f->arity[c];
  for (int c : ord) {
    const Leaf& L = net.leaves[c];
    bool ok = true;
    for (int j = 0; j < L.rank(); j++)
      if (used[f->var_of[voff[c] + j]]) ok = false;
    double mass = clause_mass(L);
    if (!ok || gain(c) <= 0) continue;
    for (int j = 0; j < L.rank(); j++) used[f->var_of[voff[c] + j]] = 1;
    picked[c] = 1;
    free_vars -= L.rank();
    lb += mass > 0 ? std::log2(mass) : -1e300;
  }
  lb += free_vars;
  for (int c = 0; c < m; c++) {
    if (picked[c]) continue;
    const Leaf& L = net.leaves[c];
    if (L.kind == LK_TABLE) {
      uint32_t mx = 0;
      for (uint32_t v : L.table) mx = std::max(mx, v);
      lb += mx > 0 ? std::log2((double)mx) : -1e300;
    }
  }
  net.log2_bound = lb < -1e200 ? -1e300 : lb;
  return TNC_OK;
}

}  // namespace tnc

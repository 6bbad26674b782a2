/*
 * tnc_oracle.c -- exact CPU oracle for tensor-network model counting.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py load this library.  It shares no
 * source, header, table or helper with the CUDA path and computes no residues:
 * every count it returns is a plain big integer.
 *
 * What it computes (Kourtis et al., "Fast counting with tensor networks"):
 *   Z = sum over all assignments of the product of the clause tensors
 *   (Eq. z with beta -> infinity, Sec. 2.1), i.e. the number of satisfying
 *   assignments, or, with open variables, the tensor of such counts indexed by
 *   the open variables (the worked example of Sec. 2.1).
 *
 * Two routes, both exact:
 *   tnco_bruteforce  -- the definition itself: enumerate all 2^n assignments.
 *   tnco_contract    -- the paper's network: one COPY tensor per variable
 *                       (Eq. var), one clause tensor per clause (Eq. or,
 *                       Eq. 1in3, ...), every occurrence a bond of dimension 2;
 *                       then pairwise contractions C = sum_shared A*B
 *                       (Sec. 2.1), all shared bonds of a pair at once
 *                       (Sec. 2.2), along a caller-given order or the paper's
 *                       tensor-greedy rule (Sec. 3.1.1: contract the connected
 *                       pair whose result has the smallest rank).
 *
 * Entries are fixed-width unsigned big integers of W 32-bit limbs (little
 * endian).  W is chosen by tnco_limbs so that no entry of any intermediate
 * tensor can exceed it: an entry counts (weighted) assignments of a subset of
 * the variables, so it is at most 2^n times the product of the clause maxima.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <limits.h>

#define TNCO_OK 0
#define TNCO_ERR_INVALID (-1)
#define TNCO_ERR_TOO_LARGE (-2)
#define TNCO_ERR_NOMEM (-3)

enum { K_1IN3 = 0, K_OR = 1, K_NAND = 2, K_TABLE = 3 };

static int popcount32(uint32_t x) {
  int c = 0;
  while (x) { c += (int)(x & 1u); x >>= 1; }
  return c;
}

/* Value of clause tensor `kind` of arity d at index idx (bit j = value on the
 * clause's j-th bond).  Eq. 1in3 (exactly one index is 1, any arity), Eq. or
 * (zero only when all indices are 0), NAND (zero only when all are 1), or an
 * explicit table. */
static uint32_t clause_value(int kind, int d, uint32_t idx, const uint32_t* tab) {
  switch (kind) {
    case K_1IN3: return popcount32(idx) == 1 ? 1u : 0u;
    case K_OR: return idx != 0 ? 1u : 0u;
    case K_NAND: return idx != ((1u << d) - 1u) ? 1u : 0u;
    case K_TABLE: return tab[idx];
    default: return 0u;
  }
}

/* bits needed by the largest value x */
static int bits_of(uint32_t x) {
  int b = 0;
  while (x) { b++; x >>= 1; }
  return b;
}

static int table_offset_check(int n_cons, const int32_t* arity, const uint8_t* kind,
                              long* off, long* total) {
  long t = 0;
  for (int c = 0; c < n_cons; c++) {
    off[c] = t;
    if (kind[c] == K_TABLE) t += 1L << arity[c];
  }
  *total = t;
  return 0;
}

/* Limbs so that 2^n_vars * prod(clause max) fits, plus one spare bit. */
int tnco_limbs(int n_vars, int n_cons, const int32_t* arity, const uint8_t* kind,
               const uint32_t* table) {
  long bits = (long)n_vars + 2;
  long t = 0;
  for (int c = 0; c < n_cons; c++) {
    if (kind[c] == K_TABLE) {
      uint32_t mx = 0;
      for (long i = 0; i < (1L << arity[c]); i++)
        if (table[t + i] > mx) mx = table[t + i];
      bits += bits_of(mx);
      t += 1L << arity[c];
    }
  }
  return (int)((bits + 31) / 32);
}

/* ---------------------------------------------------------------- bigint -- */

/* acc += a * b, truncated to W limbs (the true value always fits). */
static void big_muladd(uint32_t* acc, const uint32_t* a, const uint32_t* b, int W) {
  for (int i = 0; i < W; i++) {
    if (a[i] == 0) continue;
    uint64_t carry = 0;
    for (int j = 0; i + j < W; j++) {
      uint64_t t = (uint64_t)a[i] * b[j] + acc[i + j] + carry;
      acc[i + j] = (uint32_t)t;
      carry = t >> 32;
    }
  }
}

static int big_is_zero(const uint32_t* a, int W) {
  for (int i = 0; i < W; i++)
    if (a[i]) return 0;
  return 1;
}

/* acc = acc * s (small s), truncated */
static void big_mul_small(uint32_t* acc, uint32_t s, int W) {
  uint64_t carry = 0;
  for (int i = 0; i < W; i++) {
    uint64_t t = (uint64_t)acc[i] * s + carry;
    acc[i] = (uint32_t)t;
    carry = t >> 32;
  }
}

static void big_add(uint32_t* acc, const uint32_t* a, int W) {
  uint64_t carry = 0;
  for (int i = 0; i < W; i++) {
    uint64_t t = (uint64_t)acc[i] + a[i] + carry;
    acc[i] = (uint32_t)t;
    carry = t >> 32;
  }
}

/* ------------------------------------------------------------ brute force -- */

/* out[j*W..] for j in [0, 2^n_open): number (weight) of satisfying assignments
 * with open variable i equal to bit i of j.  Enumerates all 2^n_vars
 * assignments: the definition of Eq. z at beta -> infinity. */
int tnco_bruteforce(int n_vars, int n_cons, const int32_t* arity, const int32_t* var_of,
                    const uint8_t* kind, const uint32_t* table, int n_open,
                    const int32_t* open_vars, int W, uint32_t* out) {
  if (n_vars < 0 || n_vars > 34 || n_open < 0 || n_open > 16 || W <= 0) return TNCO_ERR_TOO_LARGE;
  long* toff = (long*)malloc(sizeof(long) * (size_t)(n_cons + 1));
  long* voff = (long*)malloc(sizeof(long) * (size_t)(n_cons + 1));
  if (!toff || !voff) { free(toff); free(voff); return TNCO_ERR_NOMEM; }
  long ttot;
  table_offset_check(n_cons, arity, kind, toff, &ttot);
  long s = 0;
  for (int c = 0; c < n_cons; c++) { voff[c] = s; s += arity[c]; }
  const long n_out = 1L << n_open;
  memset(out, 0, sizeof(uint32_t) * (size_t)n_out * (size_t)W);
  const int64_t total = (int64_t)1 << n_vars;
  int rc = TNCO_OK;
#pragma omp parallel
  {
    uint32_t* loc = (uint32_t*)calloc((size_t)n_out * (size_t)W, sizeof(uint32_t));
    uint32_t* prod = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)W);
    const int ok = (loc != NULL && prod != NULL);
    if (!ok) {
#pragma omp atomic write
      rc = TNCO_ERR_NOMEM;
    }
#pragma omp for schedule(static)
    for (int64_t x = 0; x < total; x++) {
      if (!ok) continue;
      memset(prod, 0, sizeof(uint32_t) * (size_t)W);
      prod[0] = 1;
      int zero = 0;
      for (int c = 0; c < n_cons && !zero; c++) {
        uint32_t idx = 0;
        for (int j = 0; j < arity[c]; j++)
          idx |= (uint32_t)((x >> var_of[voff[c] + j]) & 1) << j;
        uint32_t v = clause_value(kind[c], arity[c], idx, table + toff[c]);
        if (v == 0) zero = 1;
        else if (v != 1) big_mul_small(prod, v, W);
      }
      if (zero) continue;
      long j = 0;
      for (int i = 0; i < n_open; i++) j |= (long)((x >> open_vars[i]) & 1) << i;
      big_add(loc + j * W, prod, W);
    }
    if (ok) {
#pragma omp critical
      {
        for (long j = 0; j < n_out; j++) big_add(out + j * W, loc + j * W, W);
      }
    }
    free(loc);
    free(prod);
  }
  free(toff);
  free(voff);
  return rc;
}

/* ----------------------------------------------------- pairwise contraction -- */

typedef struct {
  int live;
  int rank;
  int* bond;      /* bond id on axis j; axis j is bit j of the flat index */
  uint32_t* v;    /* [2^rank][W] */
} otensor;

static int find_pos(const otensor* t, int b) {
  for (int j = 0; j < t->rank; j++)
    if (t->bond[j] == b) return j;
  return -1;
}

static int shared_count(const otensor* a, const otensor* b) {
  int s = 0;
  for (int i = 0; i < a->rank; i++)
    if (find_pos(b, a->bond[i]) >= 0) s++;
  return s;
}

/* C = sum over the shared bonds of A*B.  Output axes: A's unshared axes in
 * order, then B's unshared axes in order. */
static int contract_pair(const otensor* A, const otensor* B, otensor* C, int W, int max_rank) {
  int pa_sh[64], pb_sh[64], pa_fr[64], pb_fr[64];
  int k = 0, fa = 0, fb = 0;
  for (int i = 0; i < A->rank; i++) {
    int j = find_pos(B, A->bond[i]);
    if (j >= 0) { pa_sh[k] = i; pb_sh[k] = j; k++; }
    else pa_fr[fa++] = i;
  }
  for (int j = 0; j < B->rank; j++)
    if (find_pos(A, B->bond[j]) < 0) pb_fr[fb++] = j;
  int c = fa + fb;
  if (c > max_rank) return TNCO_ERR_TOO_LARGE;
  C->rank = c;
  C->live = 1;
  C->bond = (int*)malloc(sizeof(int) * (size_t)(c > 0 ? c : 1));
  size_t n = (size_t)1 << c;
  C->v = (uint32_t*)calloc(n * (size_t)W, sizeof(uint32_t));
  if (!C->bond || !C->v) { free(C->bond); free(C->v); return TNCO_ERR_NOMEM; }
  for (int i = 0; i < fa; i++) C->bond[i] = A->bond[pa_fr[i]];
  for (int j = 0; j < fb; j++) C->bond[fa + j] = B->bond[pb_fr[j]];
  const int64_t K = (int64_t)1 << k;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t o = 0; o < (int64_t)n; o++) {
    size_t ia0 = 0, ib0 = 0;
    for (int i = 0; i < fa; i++) ia0 |= (size_t)((o >> i) & 1) << pa_fr[i];
    for (int j = 0; j < fb; j++) ib0 |= (size_t)((o >> (fa + j)) & 1) << pb_fr[j];
    uint32_t* acc = C->v + (size_t)o * (size_t)W;
    for (int64_t q = 0; q < K; q++) {
      size_t ia = ia0, ib = ib0;
      for (int s = 0; s < k; s++) {
        size_t bit = (size_t)((q >> s) & 1);
        ia |= bit << pa_sh[s];
        ib |= bit << pb_sh[s];
      }
      const uint32_t* x = A->v + ia * (size_t)W;
      const uint32_t* y = B->v + ib * (size_t)W;
      if (big_is_zero(x, W) || big_is_zero(y, W)) continue;
      big_muladd(acc, x, y, W);
    }
  }
  return TNCO_OK;
}

/* the bonds of C now belong to C instead of A or B */
static void relabel(int* owner, int n_bonds, const otensor* C, int a, int b, int c) {
  for (int x = 0; x < C->rank; x++) {
    int bd = C->bond[x];
    if (bd >= n_bonds) continue;
    for (int e = 0; e < 2; e++)
      if (owner[2 * bd + e] == a || owner[2 * bd + e] == b) owner[2 * bd + e] = c;
  }
}

static void free_tensor(otensor* t) {
  free(t->bond);
  free(t->v);
  t->bond = NULL;
  t->v = NULL;
  t->live = 0;
}

/*
 * Exact count through the paper's tensor network.
 *   order, n_order : optional pairs (id_a, id_b) of live tensors to contract,
 *                    in sequence.  Ids: clause c -> c, variable v -> n_cons+v,
 *                    the i-th contraction's result -> n_cons+n_vars+i.
 *                    Whatever remains afterwards is contracted by the
 *                    tensor-greedy rule; disconnected leftovers are multiplied
 *                    (outer product) smallest rank first.
 *   max_rank       : refuse (TNCO_ERR_TOO_LARGE) any intermediate above it.
 *   out            : [2^n_open][W] limbs, index bit i = open variable i.
 *   stats          : optional int32[2] = {max rank seen, contractions done}.
 */
int tnco_contract(int n_vars, int n_cons, const int32_t* arity, const int32_t* var_of,
                  const uint8_t* kind, const uint32_t* table, int n_open,
                  const int32_t* open_vars, const int32_t* order, int n_order, int max_rank,
                  int W, uint32_t* out, int32_t* stats) {
  if (n_vars < 0 || n_cons < 0 || W <= 0 || n_open < 0 || n_open > 24) return TNCO_ERR_INVALID;
  if (max_rank <= 0 || max_rank > 34) max_rank = 34;
  const int n_leaf = n_cons + n_vars;
  const int cap = 2 * n_leaf + 2;
  otensor* T = (otensor*)calloc((size_t)cap, sizeof(otensor));
  int* occ = (int*)calloc((size_t)(n_vars > 0 ? n_vars : 1), sizeof(int));
  int* is_open = (int*)calloc((size_t)(n_vars > 0 ? n_vars : 1), sizeof(int));
  long* toff = (long*)malloc(sizeof(long) * (size_t)(n_cons + 1));
  if (!T || !occ || !is_open || !toff) { free(T); free(occ); free(is_open); free(toff); return TNCO_ERR_NOMEM; }
  long ttot;
  table_offset_check(n_cons, arity, kind, toff, &ttot);
  int rc = TNCO_OK;
  int max_seen = 0, steps = 0;

  /* clause tensors; bond id of occurrence (c, j) = running occurrence number */
  int bond = 0;
  long s = 0;
  for (int c = 0; c < n_cons && rc == TNCO_OK; c++) {
    int d = arity[c];
    if (d < 0 || d > 24) { rc = TNCO_ERR_INVALID; break; }
    otensor* t = &T[c];
    t->live = 1;
    t->rank = d;
    t->bond = (int*)malloc(sizeof(int) * (size_t)(d > 0 ? d : 1));
    t->v = (uint32_t*)calloc(((size_t)1 << d) * (size_t)W, sizeof(uint32_t));
    if (!t->bond || !t->v) { rc = TNCO_ERR_NOMEM; break; }
    for (int j = 0; j < d; j++) {
      int v = var_of[s + j];
      if (v < 0 || v >= n_vars) { rc = TNCO_ERR_INVALID; break; }
      t->bond[j] = bond + j;
      occ[v]++;
    }
    for (uint32_t idx = 0; idx < (1u << d); idx++)
      t->v[(size_t)idx * W] = clause_value(kind[c], d, idx, table + toff[c]);
    bond += d;
    s += d;
    if (d > max_seen) max_seen = d;
  }
  for (int i = 0; i < n_open && rc == TNCO_OK; i++) {
    if (open_vars[i] < 0 || open_vars[i] >= n_vars || is_open[open_vars[i]]) rc = TNCO_ERR_INVALID;
    else is_open[open_vars[i]] = 1 + i;
  }
  /* COPY tensors: rank = occurrences (+1 open bond).  A rank-0 COPY is the sum
   * over the variable's two values, i.e. the scalar 2. */
  if (rc == TNCO_OK) {
    int* fill = (int*)calloc((size_t)(n_vars > 0 ? n_vars : 1), sizeof(int));
    int open_bond0 = bond;
    for (int v = 0; v < n_vars && rc == TNCO_OK; v++) {
      otensor* t = &T[n_cons + v];
      int r = occ[v] + (is_open[v] ? 1 : 0);
      if (r > max_rank) { rc = TNCO_ERR_TOO_LARGE; break; }
      t->live = 1;
      t->rank = r;
      t->bond = (int*)malloc(sizeof(int) * (size_t)(r > 0 ? r : 1));
      t->v = (uint32_t*)calloc(((size_t)1 << r) * (size_t)W, sizeof(uint32_t));
      if (!t->bond || !t->v) { rc = TNCO_ERR_NOMEM; break; }
      if (r == 0) {
        t->v[0] = 2;
      } else {
        t->v[0] = 1;
        t->v[(((size_t)1 << r) - 1) * W] = 1;
      }
      if (r > max_seen) max_seen = r;
    }
    /* occurrence bonds in clause order */
    s = 0;
    for (int c = 0; c < n_cons && rc == TNCO_OK; c++) {
      for (int j = 0; j < arity[c]; j++) {
        int v = var_of[s + j];
        T[n_cons + v].bond[fill[v]++] = (int)(s + j);
      }
      s += arity[c];
    }
    for (int v = 0; v < n_vars && rc == TNCO_OK; v++)
      if (is_open[v]) T[n_cons + v].bond[fill[v]] = open_bond0 + (is_open[v] - 1);
    free(fill);
  }

  /* owner[2b], owner[2b+1]: the two tensors holding occurrence bond b */
  int n_bonds = bond;
  int* owner = (int*)malloc(sizeof(int) * (size_t)(2 * (n_bonds > 0 ? n_bonds : 1)));
  if (!owner) rc = TNCO_ERR_NOMEM;
  if (rc == TNCO_OK) {
    s = 0;
    for (int c = 0; c < n_cons; c++) {
      for (int j = 0; j < arity[c]; j++) {
        owner[2 * (s + j)] = c;
        owner[2 * (s + j) + 1] = n_cons + var_of[s + j];
      }
      s += arity[c];
    }
  }
  int n_t = n_leaf;
  /* explicit order */
  for (int i = 0; i < n_order && rc == TNCO_OK; i++) {
    int a = order[2 * i], b = order[2 * i + 1];
    if (a < 0 || b < 0 || a >= n_t || b >= n_t || a == b || !T[a].live || !T[b].live) {
      rc = TNCO_ERR_INVALID;
      break;
    }
    rc = contract_pair(&T[a], &T[b], &T[n_t], W, max_rank);
    if (rc != TNCO_OK) break;
    if (T[n_t].rank > max_seen) max_seen = T[n_t].rank;
    relabel(owner, n_bonds, &T[n_t], a, b, n_t);
    free_tensor(&T[a]);
    free_tensor(&T[b]);
    n_t++;
    steps++;
  }
  /* tensor-greedy for the rest: scan only pairs joined by a bond */
  while (rc == TNCO_OK) {
    int live = 0;
    for (int i = 0; i < n_t; i++) live += T[i].live;
    if (live <= 1) break;
    int ba = -1, bb = -1, brank = INT_MAX;
    for (int i = 0; i < n_t; i++) {
      if (!T[i].live) continue;
      for (int x = 0; x < T[i].rank; x++) {
        int b = T[i].bond[x];
        if (b >= n_bonds) continue; /* open bond */
        int j = owner[2 * b] == i ? owner[2 * b + 1] : owner[2 * b];
        if (j <= i || !T[j].live) continue;
        int k = shared_count(&T[i], &T[j]);
        int r = T[i].rank + T[j].rank - 2 * k;
        if (r < brank || (r == brank && (i < ba || (i == ba && j < bb)))) {
          brank = r; ba = i; bb = j;
        }
      }
    }
    if (ba < 0) { /* no connected pair: outer product of the two smallest */
      int r1 = INT_MAX, r2 = INT_MAX;
      for (int i = 0; i < n_t; i++) {
        if (!T[i].live) continue;
        if (T[i].rank < r1) { r2 = r1; bb = ba; r1 = T[i].rank; ba = i; }
        else if (T[i].rank < r2) { r2 = T[i].rank; bb = i; }
      }
      if (ba > bb) { int tmp = ba; ba = bb; bb = tmp; }
    }
    rc = contract_pair(&T[ba], &T[bb], &T[n_t], W, max_rank);
    if (rc != TNCO_OK) break;
    if (T[n_t].rank > max_seen) max_seen = T[n_t].rank;
    relabel(owner, n_bonds, &T[n_t], ba, bb, n_t);
    free_tensor(&T[ba]);
    free_tensor(&T[bb]);
    n_t++;
    steps++;
  }

  if (rc == TNCO_OK) {
    int root = -1;
    for (int i = 0; i < n_t; i++)
      if (T[i].live) root = i;
    const long n_out = 1L << n_open;
    memset(out, 0, sizeof(uint32_t) * (size_t)n_out * (size_t)W);
    if (root < 0) {
      out[0] = 1; /* empty formula: the empty product */
    } else {
      otensor* R = &T[root];
      int open_bond0 = 0;
      for (int c = 0; c < n_cons; c++) open_bond0 += arity[c];
      if (R->rank != n_open) rc = TNCO_ERR_INVALID;
      for (long j = 0; j < n_out && rc == TNCO_OK; j++) {
        long idx = 0;
        for (int ax = 0; ax < R->rank; ax++) {
          int i = R->bond[ax] - open_bond0; /* open bond of open variable i */
          idx |= ((j >> i) & 1L) << ax;
        }
        memcpy(out + j * W, R->v + (size_t)idx * W, sizeof(uint32_t) * (size_t)W);
      }
    }
  }
  if (stats) { stats[0] = max_seen; stats[1] = steps; }
  for (int i = 0; i < cap; i++) free_tensor(&T[i]);
  free(T);
  free(owner);
  free(occ);
  free(is_open);
  free(toff);
  return rc;
}

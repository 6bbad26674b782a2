"""Seeded synthetic #CSP instances (formulas only; no counting arithmetic).

Both the CUDA path and the CPU oracle consume the formulas made here, so this
module holds nothing of the method itself: no tensor entries, no contraction,
no counting.  It only draws clause lists from a counter-based generator
(splitmix64, Steele/Lea/Flood 2014) so that every instance is reproducible
from its seed on any machine.

Workloads (the paper's problems, Sec. 3.2):
  * monotone 1-in-3SAT clauses over three distinct variables (Eq. 1in3);
  * #Cubic-Vertex-Cover: one 2-variable OR clause per edge of a cubic graph
    (Sec. 3.2, the #2SAT form with Eq. or / Eq. var);
  * the paper's own 1-in-3 distribution: variables are the edges of a cubic
    graph and clauses its vertices, so each variable sits in two clauses
    (Sec. 3.2, Fig. 3).
Closed-form families used as pins (cycles, prisms, complete graphs) are here
too, as plain graphs.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

# Clause kinds.  The codes are shared by the C-ABI (include/tnc.h) and the
# oracle; their meaning is fixed by the paper's equations, not here.
KIND_1IN3 = 0    # Eq. 1in3, generalised to "exactly one of d" for any arity d
KIND_OR = 1      # Eq. or
KIND_NAND = 2    # not all ones (edge constraint of an independent set)
KIND_TABLE = 3   # explicit 2^d table (weighted / general clause)

MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64: x += 0x9E3779B97F4A7C15; z = mix(x).  Counter based."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, bound: int) -> int:
        """Uniform integer in [0, bound) by rejection (no modulo bias)."""
        if bound <= 0:
            raise ValueError("bound must be positive")
        limit = (1 << 64) - ((1 << 64) % bound)
        while True:
            x = self.next_u64()
            if x < limit:
                return x % bound


def derive_seed(master: int, index: int) -> int:
    """Independent per-item seed: one splitmix64 output at counter `index`."""
    g = SplitMix64((master * 0x9E3779B97F4A7C15 + index) & MASK64)
    return g.next_u64()


@dataclass
class Formula:
    """A #CSP formula: clause i constrains variables clauses[i] with kinds[i].

    open_vars lists variables whose COPY tensor carries one extra, uncontracted
    bond; the result is then a tensor over those bonds (in that order, first
    variable = least significant index bit) instead of a scalar.
    """
    n_vars: int
    clauses: List[Tuple[int, ...]]
    kinds: List[int]
    tables: List[Optional[Sequence[int]]] = field(default_factory=list)
    open_vars: List[int] = field(default_factory=list)
    name: str = ""

    def __post_init__(self):
        if not self.tables:
            self.tables = [None] * len(self.clauses)
        if len(self.kinds) != len(self.clauses) or len(self.tables) != len(self.clauses):
            raise ValueError("clauses, kinds and tables differ in length")
        for c, k, t in zip(self.clauses, self.kinds, self.tables):
            for v in c:
                if not 0 <= v < self.n_vars:
                    raise ValueError(f"variable {v} out of range")
            if k == KIND_TABLE:
                if t is None or len(t) != (1 << len(c)):
                    raise ValueError("TABLE clause needs 2^arity entries")
        for v in self.open_vars:
            if not 0 <= v < self.n_vars:
                raise ValueError(f"open variable {v} out of range")
        if len(set(self.open_vars)) != len(self.open_vars):
            raise ValueError("open variables must be distinct")

    @property
    def n_cons(self) -> int:
        return len(self.clauses)

    def flat(self):
        """(arity[], var_of[], kind[], table[]) as plain int lists (C-ABI order)."""
        arity = [len(c) for c in self.clauses]
        var_of = [v for c in self.clauses for v in c]
        table: List[int] = []
        for k, t in zip(self.kinds, self.tables):
            if k == KIND_TABLE:
                table.extend(int(x) for x in t)
        return arity, var_of, list(self.kinds), table


# ----------------------------------------------------------------------------
# graphs
# ----------------------------------------------------------------------------

def _connected(n: int, edges: Sequence[Tuple[int, int]]) -> bool:
    adj = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    seen = [False] * n
    stack = [0]
    seen[0] = True
    while stack:
        u = stack.pop()
        for w in adj[u]:
            if not seen[w]:
                seen[w] = True
                stack.append(w)
    return all(seen)


def random_cubic_graph(n: int, seed: int, max_tries: int = 100000) -> List[Tuple[int, int]]:
    """Simple connected 3-regular graph on n vertices (n even, n >= 4).

    Configuration model: 3n stubs are paired by a uniform random perfect
    matching (Fisher-Yates shuffle, then consecutive pairs); a pairing with a
    self-loop or a repeated edge, or a disconnected result, is rejected and
    redrawn.  Accepted graphs are uniform over simple cubic graphs.
    """
    if n < 4 or n % 2:
        raise ValueError("a cubic graph needs an even n >= 4")
    g = SplitMix64(seed)
    for _ in range(max_tries):
        stubs = [v for v in range(n) for _ in range(3)]
        for i in range(len(stubs) - 1, 0, -1):
            j = g.below(i + 1)
            stubs[i], stubs[j] = stubs[j], stubs[i]
        edges = []
        seen = set()
        ok = True
        for i in range(0, len(stubs), 2):
            u, v = stubs[i], stubs[i + 1]
            if u == v:
                ok = False
                break
            e = (min(u, v), max(u, v))
            if e in seen:
                ok = False
                break
            seen.add(e)
            edges.append(e)
        if ok and _connected(n, edges):
            return edges
    raise RuntimeError("no simple connected cubic graph found")


def random_planar_cubic_graph(n: int, seed: int, flips_per_edge: int = 20) -> List[Tuple[int, int]]:
    """A seeded random simple connected planar cubic graph on n vertices (n
    even, >= 4): the dual of a random triangulation of the sphere with n/2 + 2
    vertices.  The triangulation starts as a bipyramid over a cycle and is
    mixed by random edge flips (an edge ab between triangles abc and abd
    becomes cd when c and d are not adjacent and a and b keep degree >= 3);
    its triangles are the graph's vertices and two triangles sharing an edge
    are adjacent.  Flips keep the triangulation simple, so the dual is simple
    and 3-connected."""
    if n < 4 or n % 2:
        raise ValueError("a cubic graph needs an even n >= 4")
    V = n // 2 + 2
    g = SplitMix64(seed)
    top, bottom, ring = V - 2, V - 1, V - 2
    tris = []
    for i in range(ring):
        j = (i + 1) % ring
        tris.append((top, i, j))
        tris.append((bottom, j, i))
    if ring == 2:  # V = 4: the tetrahedron
        tris = [(0, 1, 2), (0, 3, 1), (1, 3, 2), (2, 3, 0)]
    for _ in range(flips_per_edge * 3 * V):
        # edge -> its two triangles
        owner = {}
        for ti, (a, b, c) in enumerate(tris):
            for u, v in ((a, b), (b, c), (c, a)):
                owner.setdefault((min(u, v), max(u, v)), []).append(ti)
        edges = sorted(owner)
        a, b = edges[g.below(len(edges))]
        t1, t2 = owner[(a, b)]
        c = [x for x in tris[t1] if x not in (a, b)][0]
        d = [x for x in tris[t2] if x not in (a, b)][0]
        deg = {}
        for u, v in edges:
            deg[u] = deg.get(u, 0) + 1
            deg[v] = deg.get(v, 0) + 1
        if c == d or (min(c, d), max(c, d)) in owner or deg[a] <= 3 or deg[b] <= 3:
            continue
        # keep the orientation: triangle t1 = (a, b, c) in some rotation
        r = tris[t1]
        k = r.index(a)
        if r[(k + 1) % 3] != b:
            a, b = b, a
        tris[t1] = (a, d, c)
        tris[t2] = (b, c, d)
    owner = {}
    for ti, (a, b, c) in enumerate(tris):
        for u, v in ((a, b), (b, c), (c, a)):
            owner.setdefault((min(u, v), max(u, v)), []).append(ti)
    return sorted((min(t), max(t)) for t in owner.values())


def cycle_graph(n: int) -> List[Tuple[int, int]]:
    return [(i, (i + 1) % n) for i in range(n)]


def prism_graph(n: int) -> List[Tuple[int, int]]:
    """Circular ladder with n rungs: two n-cycles joined by a perfect matching."""
    e = [(i, (i + 1) % n) for i in range(n)]
    e += [(n + i, n + (i + 1) % n) for i in range(n)]
    e += [(i, n + i) for i in range(n)]
    return e


def complete_graph(n: int) -> List[Tuple[int, int]]:
    return [(i, j) for i in range(n) for j in range(i + 1, n)]


def complete_bipartite(a: int, b: int) -> List[Tuple[int, int]]:
    return [(i, a + j) for i in range(a) for j in range(b)]


# ----------------------------------------------------------------------------
# formulas
# ----------------------------------------------------------------------------

def vertex_cover_formula(n: int, edges: Sequence[Tuple[int, int]], name: str = "") -> Formula:
    """#Vertex-Cover as #2SAT: a variable per vertex, an OR clause per edge."""
    return Formula(n, [tuple(e) for e in edges], [KIND_OR] * len(edges), name=name or f"vc{n}")


def independent_set_formula(n: int, edges: Sequence[Tuple[int, int]], name: str = "") -> Formula:
    """#Independent-Set: a variable per vertex, a NAND clause per edge."""
    return Formula(n, [tuple(e) for e in edges], [KIND_NAND] * len(edges), name=name or f"is{n}")


def cubic_vertex_cover(n: int, seed: int) -> Formula:
    """#Cubic-Vertex-Cover on a seeded random simple connected cubic graph."""
    return vertex_cover_formula(n, random_cubic_graph(n, seed), name=f"cubic_vc_n{n}_s{seed}")


def one_in_three(n: int, m: int, seed: int) -> Formula:
    """Monotone 1-in-3SAT: m clauses, each over 3 distinct variables drawn
    uniformly without replacement; duplicate clauses are allowed."""
    if n < 3:
        raise ValueError("need at least 3 variables")
    g = SplitMix64(seed)
    clauses = []
    for _ in range(m):
        a = g.below(n)
        b = g.below(n - 1)
        if b >= a:
            b += 1
        lo, hi = min(a, b), max(a, b)
        c = g.below(n - 2)
        if c >= lo:
            c += 1
        if c >= hi:
            c += 1
        clauses.append((a, b, c))
    return Formula(n, clauses, [KIND_1IN3] * m, name=f"1in3_n{n}_m{m}_s{seed}")


def cubic_one_in_three(n_vertices: int, seed: int) -> Formula:
    """The paper's 1-in-3 distribution: clauses are the vertices of a random
    cubic graph and variables its edges, so every variable is in 2 clauses."""
    edges = random_cubic_graph(n_vertices, seed)
    inc: List[List[int]] = [[] for _ in range(n_vertices)]
    for idx, (u, v) in enumerate(edges):
        inc[u].append(idx)
        inc[v].append(idx)
    clauses = [tuple(c) for c in inc]
    return Formula(len(edges), clauses, [KIND_1IN3] * n_vertices,
                   name=f"cubic1in3_v{n_vertices}_s{seed}")


def cnf_formula(n_vars: int, clauses: Sequence[Sequence[int]], name: str = "") -> Formula:
    """General CNF with negated literals (Sec. 2.1: a clause tensor is 1 on the
    assignments that satisfy the clause; a negated literal reverses its bond's
    index).  Literals are DIMACS-style: +(v+1) is x_v, -(v+1) is not x_v.  A
    clause becomes a TABLE tensor over its distinct variables (index bit i =
    value of the i-th), 1 everywhere except the one assignment that falsifies
    every literal; a clause with x and not x is the all-ones table."""
    cl, tabs = [], []
    for lits in clauses:
        sign = {}
        taut = False
        for lit in lits:
            if lit == 0 or abs(lit) > n_vars:
                raise ValueError(f"literal {lit} out of range")
            v, neg = abs(lit) - 1, lit < 0
            if v in sign and sign[v] != neg:
                taut = True
            sign[v] = neg
        vs = tuple(sign)
        table = [1] * (1 << len(vs))
        if not taut:
            table[sum(1 << i for i, v in enumerate(vs) if sign[v])] = 0
        cl.append(vs)
        tabs.append(table)
    return Formula(n_vars, cl, [KIND_TABLE] * len(cl), tables=tabs, name=name or f"cnf{n_vars}")


def random_k_cnf(n: int, m: int, k: int, seed: int) -> Formula:
    """m clauses of k distinct variables drawn uniformly, each literal negated
    with probability 1/2 (seeded splitmix64)."""
    g = SplitMix64(seed)
    clauses = []
    for _ in range(m):
        vs: List[int] = []
        while len(vs) < k:
            v = g.below(n)
            if v not in vs:
                vs.append(v)
        clauses.append([(v + 1) * (-1 if g.below(2) else 1) for v in vs])
    return cnf_formula(n, clauses, name=f"cnf{k}_{n}_{m}_{seed}")


def batch_one_in_three(count: int, master_seed: int, n_lo: int = 50, n_hi: int = 150,
                       d_lo: float = 0.5, d_hi: float = 0.8) -> List[Formula]:
    """Uneven batch: n ~ U{n_lo..n_hi}, m = round(n * U[d_lo, d_hi))."""
    out = []
    for i in range(count):
        s = derive_seed(master_seed, i)
        g = SplitMix64(s)
        n = n_lo + g.below(n_hi - n_lo + 1)
        d = d_lo + (d_hi - d_lo) * g.uniform()
        m = int(round(n * d))
        out.append(one_in_three(n, m, g.next_u64()))
    return out


def worked_example() -> Formula:
    """The open network of Sec. 2.1: two 3-variable OR clauses sharing two
    variables (x0, x1); y0 = variable 2 in clause 0 and y1 = variable 3 in
    clause 1 stay open.  Result index (y0 + 2*y1)."""
    return Formula(4, [(2, 0, 1), (0, 1, 3)], [KIND_OR, KIND_OR], open_vars=[2, 3],
                   name="worked_example")

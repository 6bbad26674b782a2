"""Helpers shared by the tests (random orders and formulas); no counting here."""
from paper_1805_00475_gb300 import instances as I


def random_order(rng, f):
    """A random full contraction order over connected pairs (ids as the oracle)."""
    n_leaf = f.n_cons + f.n_vars
    bonds = {}
    for c, vs in enumerate(f.clauses):
        for v in vs:
            bonds.setdefault(c, set()).add(f.n_cons + v)
            bonds.setdefault(f.n_cons + v, set()).add(c)
    live = set(range(n_leaf))
    for t in live:
        bonds.setdefault(t, set())
    nxt, order = n_leaf, []
    while len(live) > 1:
        pairs = sorted((a, b) for a in live for b in bonds[a] if b in live and a < b)
        a, b = rng.choice(pairs) if pairs else tuple(sorted(rng.sample(sorted(live), 2)))
        order.append((a, b))
        nb = (bonds[a] | bonds[b]) - {a, b}
        for x in nb:
            bonds[x] -= {a, b}
            bonds[x].add(nxt)
        bonds[nxt] = nb
        live -= {a, b}
        live.add(nxt)
        nxt += 1
    return order


def random_formula(rng, n, m, n_open=0, weights=(0, 1, 2, 3, 4, 5), allow_empty=False):
    """Random clauses of every kind (arity 1..4, TABLE weights from `weights`)."""
    clauses, kinds, tables = [], [], []
    for _ in range(m):
        d = rng.randint(0 if (allow_empty and rng.random() < 0.05) else 1, 4)
        vs = tuple(rng.sample(range(n), min(d, n)))
        k = rng.choice([I.KIND_1IN3, I.KIND_OR, I.KIND_NAND, I.KIND_TABLE])
        clauses.append(vs)
        kinds.append(k)
        tables.append([rng.choice(weights) for _ in range(1 << len(vs))] if k == I.KIND_TABLE else None)
    return I.Formula(n, clauses, kinds, tables, open_vars=rng.sample(range(n), n_open))

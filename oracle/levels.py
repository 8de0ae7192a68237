"""Oracle: the MTP basis set enumerated from its definition (Sec. 2.1, Eqs. 5-6).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module;
only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.

What the paper fixes (Sec. 2.1):
  * a moment M_{mu,nu} is a rank-nu symmetric tensor with level 2 + 4 mu + nu (Eq. 5);
  * the level of a product or contraction of moments is the sum of their levels;
  * every scalar obtainable by contracting one or more moments is a basis function B_alpha,
    and the basis holds all of them with lev B_alpha <= lev_max (example: Eq. 6, nine
    functions at lev_max = 8).

Representation used here: a basis function is a loopless multigraph.  Each node is a moment
(mu, nu); each edge is one index of one node summed against one index of another node, so a
node of rank nu has degree nu.  A graph with several connected components is the product of
the component scalars.  Self-contractions (traces, a loop) are excluded: the lev_max = 8 list
of Eq. 6 has no tr M_{0,2} although its level (4) is admissible.  Products of separate
contractions are included: M_{0,0}^2 and M_{0,0} (M_{0,1} . M_{0,1}) are in Eq. 6.

Canonical form (shared *definition* with the GPU-side generator; the code is separate):
  component code for a node order pi:
      [n, mu_pi0, nu_pi0, ..., mu_pi(n-1), nu_pi(n-1), A[pi_i][pi_j] for i<j row-major]
  the canonical code is the lexicographic minimum over all n! orders.
  components are numbered by the key (level, n, canonical code);
  a basis function is the ascending tuple of its component numbers; basis functions are
  ordered by the key (level, total number of moments, component-number tuple).

Ordering is this build's own reading (the paper's list in Eq. 6 is not level-sorted).
"""

from __future__ import annotations

import itertools
from dataclasses import dataclass
from functools import lru_cache


def moment_level(mu: int, nu: int) -> int:
    """Eq. 5: lev M_{mu,nu} = 2 + 4 mu + nu."""
    return 2 + 4 * mu + nu


@dataclass(frozen=True)
class Component:
    """One connected contraction: canonical node labels and adjacency (upper triangle)."""

    labels: tuple  # ((mu, nu), ...) in canonical order
    adj: tuple  # A[i][j], i < j, row-major, canonical order

    @property
    def n(self) -> int:
        return len(self.labels)

    @property
    def level(self) -> int:
        return sum(moment_level(mu, nu) for mu, nu in self.labels)

    def code(self) -> tuple:
        flat = [self.n]
        for mu, nu in self.labels:
            flat += [mu, nu]
        return tuple(flat) + tuple(self.adj)

    def matrix(self):
        n = self.n
        a = [[0] * n for _ in range(n)]
        k = 0
        for i in range(n):
            for j in range(i + 1, n):
                a[i][j] = a[j][i] = self.adj[k]
                k += 1
        return a


def _upper(a, order):
    n = len(order)
    return tuple(a[order[i]][order[j]] for i in range(n) for j in range(i + 1, n))


def _label_sorting_orders(labels):
    """Every node order that lists the labels in ascending order.

    The label part of the code precedes the adjacency part, so the lexicographic minimum over
    all n! orders is always reached by an order of this kind; the others need not be tried."""
    n = len(labels)
    idx = sorted(range(n), key=lambda k: labels[k])
    groups = [list(g) for _, g in itertools.groupby(idx, key=lambda k: labels[k])]
    for parts in itertools.product(*[itertools.permutations(g) for g in groups]):
        yield tuple(k for part in parts for k in part)


def canonical_component(labels, a) -> Component:
    """Lexicographic minimum of the component code over every node order."""
    n = len(labels)
    best = None
    for order in _label_sorting_orders(labels):
        code = [n]
        for k in order:
            code += [labels[k][0], labels[k][1]]
        code = tuple(code) + _upper(a, order)
        if best is None or code < best[0]:
            best = (code, order)
    order = best[1]
    return Component(tuple(labels[k] for k in order), _upper(a, order))


def _connected(a) -> bool:
    n = len(a)
    seen = {0}
    stack = [0]
    while stack:
        u = stack.pop()
        for v in range(n):
            if a[u][v] and v not in seen:
                seen.add(v)
                stack.append(v)
    return len(seen) == n


def _adjacency_with_degrees(deg):
    """Every symmetric non-negative integer matrix with zero diagonal and row sums deg."""
    n = len(deg)
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    a = [[0] * n for _ in range(n)]
    left = list(deg)

    def rec(p):
        if p == len(pairs):
            if all(x == 0 for x in left):
                yield [row[:] for row in a]
            return
        i, j = pairs[p]
        # once every pair touching i has been assigned, i must be saturated
        last_for_i = all(q[0] != i and q[1] != i for q in pairs[p + 1:])
        lo = left[i] if last_for_i else 0
        for m in range(lo, min(left[i], left[j]) + 1):
            a[i][j] = a[j][i] = m
            left[i] -= m
            left[j] -= m
            yield from rec(p + 1)
            left[i] += m
            left[j] += m
        a[i][j] = a[j][i] = 0

    yield from rec(0)


@lru_cache(maxsize=None)
def connected_components(lev_max: int):
    """All connected contractions with level <= lev_max, sorted by (level, n, code)."""
    found = set()
    # a single node is a scalar only when nu = 0 (a rank >= 1 node alone needs a trace)
    mu = 0
    while moment_level(mu, 0) <= lev_max:
        found.add(Component(((mu, 0),), ()))
        mu += 1
    # n >= 2 nodes: every node has nu >= 1 (a scalar node cannot be connected to anything)
    labels_all = [(mu, nu) for mu in range(lev_max) for nu in range(1, lev_max)
                  if moment_level(mu, nu) <= lev_max]
    labels_all.sort()

    def label_multisets(n, start, budget):
        """Ascending label lists of length n whose levels sum to at most budget."""
        if n == 0:
            yield []
            return
        for k in range(start, len(labels_all)):
            lv = moment_level(*labels_all[k])
            if lv + 3 * (n - 1) <= budget:  # every further node costs at least 3
                for rest in label_multisets(n - 1, k, budget - lv):
                    yield [labels_all[k]] + rest

    n = 2
    while 3 * n <= lev_max:
        for labels in label_multisets(n, 0, lev_max):
            deg = [nu for _, nu in labels]
            if sum(deg) % 2:
                continue
            for a in _adjacency_with_degrees(deg):
                if _connected(a):
                    found.add(canonical_component(list(labels), a))
        n += 1
    return tuple(sorted(found, key=lambda c: (c.level, c.n, c.code())))


@dataclass(frozen=True)
class BasisFunction:
    components: tuple  # ascending component numbers
    level: int
    n_moments: int


@lru_cache(maxsize=None)
def basis(lev_max: int):
    """All basis functions with level <= lev_max in canonical order (Sec. 2.1)."""
    comps = connected_components(lev_max)
    out = []

    def rec(start, chosen, level):
        if chosen:
            out.append(BasisFunction(tuple(chosen), level,
                                     sum(comps[k].n for k in chosen)))
        for k in range(start, len(comps)):
            lv = level + comps[k].level
            if lv <= lev_max:
                chosen.append(k)
                rec(k, chosen, lv)
                chosen.pop()

    rec(0, [], 0)
    out.sort(key=lambda b: (b.level, b.n_moments, b.components))
    return tuple(out)


def used_moments(lev_max: int):
    """Moments (mu, nu) that occur in at least one basis function, sorted by (mu, nu)."""
    used = set()
    for c in connected_components(lev_max):
        used.update(c.labels)
    return tuple(sorted(used))


def level_table(lev_max: int):
    """Flat int list describing the basis (the canonical level table).

    Layout: [m, then for each basis function: level, number of components,
    then for each component: n, mu_0, nu_0, ..., A upper triangle]."""
    comps = connected_components(lev_max)
    bl = basis(lev_max)
    flat = [len(bl)]
    for b in bl:
        flat += [b.level, len(b.components)]
        for k in b.components:
            flat += list(comps[k].code())
    return flat


def describe(b: BasisFunction, lev_max: int) -> str:
    """Readable name such as 'M00*M01.M01' (used by the golden-file test)."""
    comps = connected_components(lev_max)
    parts = []
    for k in b.components:
        c = comps[k]
        names = [f"M{mu}{nu}" for mu, nu in c.labels]
        if c.n == 1:
            parts.append(names[0])
        else:
            a = c.matrix()
            edges = [f"{i}-{j}x{a[i][j]}" for i in range(c.n) for j in range(i + 1, c.n) if a[i][j]]
            parts.append("(" + ",".join(names) + ";" + ",".join(edges) + ")")
    return "*".join(parts)

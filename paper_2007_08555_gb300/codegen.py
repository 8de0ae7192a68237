"""Build-time generator of the per-level tables and unrolled CUDA code of the MTP kernels.

For a maximum level L it derives, from the basis definition of Sec. 2.1 (Eqs. 5-6):

* the basis set: every scalar contraction of moments M_{mu,nu} (level 2 + 4 mu + nu) with total
  level <= L, as loopless multigraphs (node = moment, edge = one contracted index pair),
  products of connected contractions included;
* the canonical level table (int32), in the order and format documented in include/mtp.h, so the
  library's table can be compared bit for bit with an independent enumeration;
* the moment components: for every moment in use, one entry per monomial x^a y^b z^c
  (a + b + c = nu); symmetric storage of M_{mu,nu};
* a contraction program: every connected contraction is evaluated as a sequence of pairwise
  merges of sub-networks.  A merged sub-network S is a tensor whose open indices are grouped by
  the node they belong to; inside a group the tensor is symmetric, so it is stored by monomial.
  Merging S1 and S2 over the edge bundles (u in S1, v in S2, multiplicity h) sums, for every
  bundle, over the monomials of degree h weighted by their multinomial count h!/(a! b! c!).
  Every output entry is therefore a sum of terms  w * val[i] * val[j]  ("ops").  Identical
  sub-networks are shared between contractions, merge orders are chosen by dynamic programming
  over connected subsets to minimise the number of ops;
* the ops arranged in dependency layers and spread over the 32 lanes of a warp, for the forward
  and the adjoint (reverse-mode) pass;
* unrolled per-slice code for the thread-per-atom moment and force kernels.

Nothing here is shared with the test oracle; the canonical order is a documented convention.
"""

from __future__ import annotations

import itertools
import math
import os
from collections import defaultdict
from dataclasses import dataclass, field

SUPPORTED_LEVELS = tuple(range(2, 22, 2))
WARP = 32


def mlevel(mu, nu):
    return 2 + 4 * mu + nu


def monomials(g):
    """Monomials (a, b, c) of degree g: a descending, then b descending."""
    return [(a, b, g - a - b) for a in range(g, -1, -1) for b in range(g - a, -1, -1)]


def mono_index(m):
    a, b, c = m
    g = a + b + c
    return monomials(g).index(m)


def n_monomials(g):
    return (g + 1) * (g + 2) // 2


def multinomial(m):
    a, b, c = m
    return math.factorial(a + b + c) // (math.factorial(a) * math.factorial(b) * math.factorial(c))


# ---------------------------------------------------------------------------------------------
# Basis enumeration (stub pairing + canonical code)
# ---------------------------------------------------------------------------------------------
def _code(labels, adj, order):
    n = len(order)
    out = [n]
    for k in order:
        out.extend(labels[k])
    for x in range(n):
        for y in range(x + 1, n):
            out.append(adj[order[x]][order[y]])
    return tuple(out)


def canonical(labels, adj):
    """(code, order): lexicographically smallest code over node orders.  Orders that do not sort
    the labels ascending cannot win (labels precede the adjacency in the code)."""
    n = len(labels)
    by_label = defaultdict(list)
    for k in range(n):
        by_label[tuple(labels[k])].append(k)
    keys = sorted(by_label)
    best = None
    for choice in itertools.product(*[list(itertools.permutations(by_label[k])) for k in keys]):
        order = [x for part in choice for x in part]
        code = _code(labels, adj, order)
        if best is None or code < best[0]:
            best = (code, order)
    return best


def _pairings(stubs, n):
    """Yield adjacency matrices from matching node stubs pairwise (no loops), deduplicated."""
    seen = set()

    def rec(rest, adj):
        if not rest:
            key = tuple(tuple(r) for r in adj)
            if key not in seen:
                seen.add(key)
                yield [r[:] for r in adj]
            return
        u = rest[0]
        tried = set()
        for k in range(1, len(rest)):
            v = rest[k]
            if v == u or v in tried:
                continue
            tried.add(v)
            adj[u][v] += 1
            adj[v][u] += 1
            yield from rec(rest[1:k] + rest[k + 1:], adj)
            adj[u][v] -= 1
            adj[v][u] -= 1

    yield from rec(stubs, [[0] * n for _ in range(n)])


def _is_connected(adj):
    n = len(adj)
    seen, todo = {0}, [0]
    while todo:
        u = todo.pop()
        for v in range(n):
            if adj[u][v] and v not in seen:
                seen.add(v)
                todo.append(v)
    return len(seen) == n


def enumerate_components(L):
    """Connected contractions with level <= L as {code: (labels, adj)} (labels/adj in canonical order)."""
    comps = {}
    for mu in range(L):
        if mlevel(mu, 0) <= L:
            comps[(1, mu, 0)] = ([(mu, 0)], [[0]])
    pool = sorted((mu, nu) for mu in range(L) for nu in range(1, L) if mlevel(mu, nu) <= L)

    def grow(start, labels, lev):
        if len(labels) >= 2 and sum(nu for _, nu in labels) % 2 == 0:
            stubs = [k for k, (_, nu) in enumerate(labels) for _ in range(nu)]
            for adj in _pairings(stubs, len(labels)):
                if _is_connected(adj):
                    code, order = canonical(labels, adj)
                    if code not in comps:
                        comps[code] = ([labels[k] for k in order],
                                       [[adj[order[x]][order[y]] for y in range(len(order))]
                                        for x in range(len(order))])
        for k in range(start, len(pool)):
            if lev + mlevel(*pool[k]) <= L:
                grow(k, labels + [pool[k]], lev + mlevel(*pool[k]))

    grow(0, [], 0)
    return comps


@dataclass
class Basis:
    L: int
    comps: list  # [(code, labels, adj, level)] sorted by (level, n, code)
    funcs: list  # [(level, n_moments, tuple(component ids))] canonical order

    @property
    def m(self):
        return len(self.funcs)


def build_basis(L) -> Basis:
    raw = enumerate_components(L)
    comps = []
    for code, (labels, adj) in raw.items():
        comps.append((code, labels, adj, sum(mlevel(*x) for x in labels)))
    comps.sort(key=lambda t: (t[3], len(t[1]), t[0]))
    funcs = []
    stack = [((), 0, 0, 0)]
    while stack:
        ids, lev, nm, start = stack.pop()
        if ids:
            funcs.append((lev, nm, ids))
        for k in range(start, len(comps)):
            if lev + comps[k][3] <= L:
                stack.append((ids + (k,), lev + comps[k][3], nm + len(comps[k][1]), k))
    funcs.sort()
    return Basis(L, comps, funcs)


def level_table(basis: Basis):
    out = [basis.m]
    for lev, _, ids in basis.funcs:
        out += [lev, len(ids)]
        for k in ids:
            out += list(basis.comps[k][0])
    return out


# ---------------------------------------------------------------------------------------------
# Contraction program
# ---------------------------------------------------------------------------------------------
@dataclass
class Program:
    L: int
    basis: Basis
    moments: list  # used (mu, nu), sorted
    comp_list: list  # moment components [(mu, (a, b, c))] in storage order
    comp_index: dict  # (mu, (a,b,c)) -> index
    n_values: int = 0
    ops: list = field(default_factory=list)  # (k, i, j, w) in creation order
    basis_value: list = field(default_factory=list)  # value index of each basis function
    n_mu: int = 0
    numax: int = 0


class _Builder:
    def __init__(self, basis: Basis):
        self.basis = basis
        L = basis.L
        used = set()
        for _, labels, _, _ in basis.comps:
            used.update(tuple(x) for x in labels)
        self.moments = sorted(used)
        numax = max(nu for _, nu in self.moments)
        n_mu = max(mu for mu, _ in self.moments) + 1
        # components ordered by monomial (degree, index) then mu: a slice of monomials holds all
        # of their radial channels
        comp_list = []
        for g in range(numax + 1):
            for m in monomials(g):
                for mu in range(n_mu):
                    if (mu, g) in used:
                        comp_list.append((mu, m))
        self.prog = Program(L, basis, self.moments, comp_list, {c: k for k, c in enumerate(comp_list)},
                            n_mu=n_mu, numax=numax)
        self.n_values = len(comp_list)
        self.ops = []
        self.tensors = {}  # canonical key -> (order of nodes as (label, open) list, base index, group sizes)

    # a sub-network: labels per node, internal adjacency, open index count per node
    def _key(self, labels, adj, open_):
        lab2 = [(labels[k][0], labels[k][1], open_[k]) for k in range(len(labels))]
        code, order = canonical(lab2, adj)
        return code, order

    def _entries(self, open_):
        size = 1
        for g in open_:
            if g > 0:
                size *= n_monomials(g)
        return size

    def _entry_index(self, open_, monos):
        """Mixed-radix index over the groups with g > 0 (first group most significant)."""
        idx = 0
        for g, m in zip(open_, monos):
            if g > 0:
                idx = idx * n_monomials(g) + mono_index(m)
        return idx

    def tensor(self, labels, adj, open_):
        """Value base index of the (shared) tensor of a sub-network, building it if needed.
        Returns (base, order) with order mapping canonical position -> local node."""
        n = len(labels)
        if n == 1:
            return None, [0]
        code, order = self._key(labels, adj, open_)
        if code in self.tensors:
            return self.tensors[code], order
        raise KeyError(code)

    def value_of(self, labels, adj, open_, order_base, monos_local):
        """Value index of one entry of a sub-network tensor, monos given per local node."""
        n = len(labels)
        if n == 1:
            return self.prog.comp_index[(labels[0][0], monos_local[0])]
        base, order = order_base
        open_c = [open_[k] for k in order]
        monos_c = [monos_local[k] for k in order]
        return base + self._entry_index(open_c, monos_c)

    def build(self):
        for code, labels, adj, lev in self.basis.comps:
            if len(labels) > 1:
                self._build_component(labels, adj)
        comp_value = []
        for code, labels, adj, lev in self.basis.comps:
            if len(labels) == 1:
                comp_value.append(self.prog.comp_index[(labels[0][0], (0, 0, 0))])
            else:
                base, _ = self.tensor(labels, adj, [0] * len(labels))
                comp_value.append(base)
        # basis functions: single components map to the component value; a product of k components
        # is (the basis function of its first k-1 components) * (its last component)
        func_value = {}
        out = []
        for lev, nm, ids in self.basis.funcs:
            if len(ids) == 1:
                v = comp_value[ids[0]]
            else:
                v = self.n_values
                self.n_values += 1
                self.ops.append((v, func_value[ids[:-1]], comp_value[ids[-1]], 1.0))
            func_value[ids] = v
            out.append(v)
        self.prog.basis_value = out
        self.prog.ops = self.ops
        self.prog.n_values = self.n_values
        return self.prog

    # -- dynamic programme over connected subsets of one component --------------------------
    def _build_component(self, labels, adj):
        n = len(labels)
        nu = [x[1] for x in labels]

        def connected(S):
            S = list(S)
            seen, todo = {S[0]}, [S[0]]
            while todo:
                u = todo.pop()
                for v in S:
                    if adj[u][v] and v not in seen:
                        seen.add(v)
                        todo.append(v)
            return len(seen) == len(S)

        def sub(S):
            S = sorted(S)
            lab = [labels[u] for u in S]
            a = [[adj[u][v] for v in S] for u in S]
            op = [nu[u] - sum(adj[u][w] for w in S) for u in S]
            return S, lab, a, op

        memo = {}

        def cost(S):
            S = frozenset(S)
            if len(S) == 1:
                return 0, None
            if S in memo:
                return memo[S]
            Sl, lab, a, op = sub(S)
            code, _ = self._key(lab, a, op)
            if code in self.tensors:
                memo[S] = (0, None)
                return memo[S]
            best = None
            first = min(S)
            for r in range(1, len(S)):
                for S1 in itertools.combinations(sorted(S), r):
                    if first not in S1:
                        continue
                    S1 = frozenset(S1)
                    S2 = S - S1
                    if not connected(S1) or not connected(S2):
                        continue
                    if not any(adj[u][v] for u in S1 for v in S2):
                        continue
                    c = self._entries(op)
                    for u in S1:
                        for v in S2:
                            if adj[u][v]:
                                c *= n_monomials(adj[u][v])
                    c1, _ = cost(S1)
                    c2, _ = cost(S2)
                    tot = c + c1 + c2
                    if best is None or tot < best[0]:
                        best = (tot, (S1, S2))
            memo[S] = best
            return best

        def realise(S):
            S = frozenset(S)
            if len(S) == 1:
                return
            Sl, lab, a, op = sub(S)
            code, order = self._key(lab, a, op)
            if code in self.tensors:
                return
            _, split = cost(S)
            S1, S2 = split
            realise(S1)
            realise(S2)
            self._merge(Sl, lab, a, op, code, order, S1, S2, labels, adj)

        cost(range(n))
        realise(range(n))

    def _merge(self, Sl, lab, a, op, code, order, S1, S2, labels, adj):
        base = self.n_values
        self.tensors[code] = base
        size = self._entries(op)
        self.n_values += size
        nu = [x[1] for x in labels]
        S1l, S2l = sorted(S1), sorted(S2)

        def handle(Sx):
            Sx_l = sorted(Sx)
            lab_x = [labels[u] for u in Sx_l]
            a_x = [[adj[u][v] for v in Sx_l] for u in Sx_l]
            op_x = [nu[u] - sum(adj[u][w] for w in Sx_l) for u in Sx_l]
            if len(Sx_l) == 1:
                return Sx_l, lab_x, a_x, op_x, None
            code_x, order_x = self._key(lab_x, a_x, op_x)
            return Sx_l, lab_x, a_x, op_x, (self.tensors[code_x], order_x)

        h1 = handle(S1)
        h2 = handle(S2)
        bundles = [(u, v, adj[u][v]) for u in S1l for v in S2l if adj[u][v]]
        # output entries: canonical order of this tensor's groups
        open_c = [op[k] for k in order]
        nodes_c = [Sl[k] for k in order]
        group_monos = [monomials(g) if g > 0 else [(0, 0, 0)] for g in open_c]
        bundle_monos = [monomials(h) for (_, _, h) in bundles]
        for out_monos in itertools.product(*group_monos):
            out_of = dict(zip(nodes_c, out_monos))
            k = base + self._entry_index(open_c, list(out_monos))
            for bm in itertools.product(*bundle_monos):
                w = 1
                tot = {u: list(out_of[u]) for u in Sl}
                for (u, v, h), m in zip(bundles, bm):
                    w *= multinomial(m)
                    for t in range(3):
                        tot[u][t] += m[t]
                        tot[v][t] += m[t]
                i = self.value_of(h1[1], h1[2], h1[3], h1[4], [tuple(tot[u]) for u in h1[0]])
                j = self.value_of(h2[1], h2[2], h2[3], h2[4], [tuple(tot[u]) for u in h2[0]])
                self.ops.append((k, i, j, float(w)))


def build_program(L) -> Program:
    return _Builder(build_basis(L)).build()


# ---------------------------------------------------------------------------------------------
# Warp layout of the forward and adjoint programs
# ---------------------------------------------------------------------------------------------
def _lane_layers(groups_by_layer):
    """groups_by_layer: list of layers, each a list of (target, [terms]).  Returns per layer a
    list of 32 lane queues (longest-processing-time greedy)."""
    out = []
    for groups in groups_by_layer:
        lanes = [[] for _ in range(WARP)]
        load = [0] * WARP
        for tgt, terms in sorted(groups, key=lambda g: -len(g[1])):
            k = min(range(WARP), key=lambda x: load[x])
            lanes[k].append((tgt, terms))
            load[k] += len(terms)
        out.append(lanes)
    return out


def forward_layout(prog: Program):
    C = len(prog.comp_list)
    depth = [0] * prog.n_values
    by_k = defaultdict(list)
    for (k, i, j, w) in prog.ops:
        by_k[k].append((i, j, w))
    for k in sorted(by_k):  # creation order is topological (inputs have smaller indices)
        depth[k] = 1 + max(max(depth[i], depth[j]) for i, j, _ in by_k[k])
    layers = defaultdict(list)
    for k, terms in by_k.items():
        layers[depth[k]].append((k, terms))
    assert all(k >= C for k in by_k)
    return _lane_layers([layers[d] for d in sorted(layers)])


def adjoint_layout(prog: Program):
    """Reverse pass: adj[t] = seed[t] + sum over ops consuming t of w * val[other] * adj[k]."""
    contrib = defaultdict(list)
    for (k, i, j, w) in prog.ops:
        contrib[i].append((j, k, w))
        contrib[j].append((i, k, w))
    consumers = defaultdict(set)
    for (k, i, j, w) in prog.ops:
        consumers[i].add(k)
        consumers[j].add(k)
    rdepth = {}

    def rd(v):
        if v in rdepth:
            return rdepth[v]
        r = 0 if not consumers[v] else 1 + max(rd(k) for k in consumers[v])
        rdepth[v] = r
        return r

    import sys
    sys.setrecursionlimit(100000)
    for v in range(prog.n_values - 1, -1, -1):
        rd(v)
    layers = defaultdict(list)
    for t, terms in contrib.items():
        layers[rdepth[t]].append((t, terms))
    return _lane_layers([layers[d] for d in sorted(layers)])


def encode_layout(layout):
    """Flatten lanes into steps: rows of 32 entries (i, j, k, flags, w).
    flags bit0: first term of a target (accumulator starts from the target's seed);
          bit1: last term (store the accumulator); bit2: padding (no work)."""
    rows = []
    layer_rows = []
    for lanes in layout:
        start = len(rows)
        seqs = []
        for lane in lanes:
            seq = []
            for tgt, terms in lane:
                for t, (a, b, w) in enumerate(terms):
                    flags = (1 if t == 0 else 0) | (2 if t == len(terms) - 1 else 0)
                    seq.append((a, b, tgt, flags, w))
            seqs.append(seq)
        steps = max((len(s) for s in seqs), default=0)
        for s in range(steps):
            row = []
            for lane in range(WARP):
                if s < len(seqs[lane]):
                    row.append(seqs[lane][s])
                else:
                    row.append((0, 0, 0, 4, 0.0))
            rows.append(row)
        layer_rows.append((start, len(rows)))
    return rows, layer_rows


# ---------------------------------------------------------------------------------------------
# Slices of the thread-per-atom kernels
# ---------------------------------------------------------------------------------------------
def slices(prog: Program, max_comps):
    """Contiguous groups of monomials (with all their radial channels) of <= max_comps components."""
    groups = []
    cur, cur_n = [], 0
    by_mono = defaultdict(list)
    order = []
    for idx, (mu, m) in enumerate(prog.comp_list):
        if m not in by_mono:
            order.append(m)
        by_mono[m].append(idx)
    for m in order:
        k = len(by_mono[m])
        if cur and cur_n + k > max_comps:
            groups.append(cur)
            cur, cur_n = [], 0
        cur.append(m)
        cur_n += k
    if cur:
        groups.append(cur)
    return [(g, [i for m in g for i in by_mono[m]]) for g in groups]


def moment_slices(prog: Program, max_comps):
    """Slices of the float moments kernel: as few as slices(prog, max_comps) gives, with their sizes
    balanced (the largest slice sets the running sums held per thread, hence the registers and the
    resident warps of the kernel).  The pair-gradient and tangent kernels keep slices(prog,
    max_comps)."""
    n = len(slices(prog, max_comps))
    C = len(prog.comp_list)
    for cap in range(-(-C // n), max_comps + 1):
        s = slices(prog, cap)
        if len(s) == n:
            return s
    return slices(prog, max_comps)


def _mono_name(m):
    return "m%d_%d_%d" % m


def _mono_code(needed, T):
    """Statements computing every monomial in `needed` (closed under parents) from x, y, z."""
    lines = []
    done = {(0, 0, 0)}
    for m in sorted(needed, key=lambda t: (sum(t), monomials(sum(t)).index(t))):
        if m in done:
            continue
        a, b, c = m
        if a > 0:
            parent, var = (a - 1, b, c), "x"
        elif b > 0:
            parent, var = (a, b - 1, c), "y"
        else:
            parent, var = (a, b, c - 1), "z"
        if parent == (0, 0, 0):
            lines.append(f"const {T} {_mono_name(m)} = {var};")
        else:
            lines.append(f"const {T} {_mono_name(m)} = {_mono_name(parent)} * {var};")
        done.add(m)
    return lines


def _closure(monos):
    need = set()
    for m in monos:
        cur = m
        while cur != (0, 0, 0):
            need.add(cur)
            a, b, c = cur
            cur = (a - 1, b, c) if a > 0 else ((a, b - 1, c) if b > 0 else (a, b, c - 1))
    return need


# Float adjoints from this level on sum their gradient terms per (direction, exponent) and per radial
# channel (_grad_terms_folded): measured on GB300 at lev_max 20, 10% fewer instructions and 7% less
# time in the pair-gradient kernel (126 registers either way).  At lev_max 16 the extra partial sums
# cost registers (124 instead of 72 per thread with eight lanes per atom) and the time was unchanged
# within the run-to-run spread, so lower levels keep one multiplication per term.
FOLD_GRAD_MIN_LEVEL = 18


def _grad_terms_folded(monos, by_m):
    """Gradient terms sum_m alpha_m grad(m) of the float adjoint with fewer multiplications.
    d/dx_d of x^a y^b z^c is e_d times a monomial of one degree less (e_d = a, b or c), so the terms
    are summed per (direction d, exponent e_d) and each partial sum is scaled by e_d once at the end,
    instead of once per term.  A monomial carried by one radial channel mu alone adds adj * mono' to
    a sum kept per (d, e_d, mu), which is scaled by f_mu once at the end, instead of forming
    alpha_m = adj f_mu for it.  Monomials of several channels form alpha_m = sum_mu adj f_mu as
    usual.  Same sum, reassociated: only the rounding differs."""
    names = ("gx", "gy", "gz")
    acc = {}  # (direction, exponent, mu or None) -> accumulator name

    def acc_name(d, e, mu):
        key = (d, e, mu)
        if key not in acc:
            acc[key] = f"{names[d]}_{e}" + ("" if mu is None else f"_f{mu}")
        return acc[key]

    body = []
    for m in monos:
        if m == (0, 0, 0):
            continue
        terms = by_m[m]
        dirs = [d for d in range(3) if m[d] > 0]

        def src_of(d):
            mm = list(m)
            mm[d] -= 1
            mm = tuple(mm)
            return None if mm == (0, 0, 0) else _mono_name(mm)

        if len(terms) == 1:
            t, mu = terms[0]
            for d in dirs:
                src = src_of(d)
                body.append(f"{acc_name(d, m[d], mu)} += " + (f"adj[{t}]" if src is None else f"adj[{t}] * {src}")
                            + ";")
            continue
        al = " + ".join(f"adj[{t}] * f[{mu}]" for t, mu in terms)
        body.append(f"{{ const T al = {al};")
        for d in dirs:
            src = src_of(d)
            term = "al" if src is None else f"al * {src}"
            if m[d] == 1:
                body.append(f"  {names[d]} += {term};")
            else:
                body.append(f"  {acc_name(d, m[d], None)} += {term};")
        body.append("}")
    decl = [f"T {v} = T(0);" for v in acc.values()]
    fin = []
    for d in range(3):
        plain = sorted(e for (dd, e, mu) in acc if dd == d and mu is None)
        if plain:
            fin.append(f"{names[d]} += " + " + ".join(f"T({e}) * {acc[(d, e, None)]}" for e in plain) + ";")
        for mu in sorted({mu for (dd, e, mu) in acc if dd == d and mu is not None}):
            es = sorted(e for (dd, e, m2) in acc if dd == d and m2 == mu)
            inner = " + ".join(acc[(d, e, mu)] if e == 1 else f"T({e}) * {acc[(d, e, mu)]}" for e in es)
            fin.append(f"{names[d]} += f[{mu}] * ({inner});")
    return decl + body + fin


def _mom_function(prog: Program, monos, comps):
    """mom(x, y, z, f, acc) of one slice: acc[t] += f[mu] x^a y^b z^c for its components (Eq. 5 for
    one neighbour)."""
    out = ["  template <class T> static __device__ __forceinline__ void mom(const T x, const T y, const T z, "
           "const T* __restrict__ f, T* __restrict__ acc) {"]
    out += ["    " + l for l in _mono_code(_closure(monos), "T")]
    for t, ci in enumerate(comps):
        mu, m = prog.comp_list[ci]
        mv = "T(1)" if m == (0, 0, 0) else _mono_name(m)
        out.append(f"    acc[{t}] += f[{mu}] * {mv};")
    out.append("  }")
    return out


def emit_slice_functions(prog: Program, slc, tag, slot_begin=None):
    """Specialisations Slice<tag><S> for every slice S (a list of (monomials, component indices)):
       mom(x,y,z,f,acc):   acc[t] += f[mu] * x^a y^b z^c                    (moments, Sec. 2.1)
       grad(x,y,z,f,df,adj,s,gx,gy,gz):
             s += sum adj * df[mu] * mono;  g += sum adj * f[mu] * grad(mono)   (adjoint)"""
    name = {"f": "SliceF", "d": "SliceD", "mf": "SliceMF"}[tag]
    out = [f"template <int S> struct {name};"]
    for si, (monos, comps) in enumerate(slc):
        out.append(f"template <> struct {name}<{si}> {{")
        out.append(f"  static constexpr int BEGIN = {min(comps)}, SIZE = {len(comps)};")
        if tag == "mf":  # the moments kernel's slices: the accumulation alone
            out += _mom_function(prog, monos, comps)
            out.append("};")
            continue
        if slot_begin is not None:
            # dV/dM of this slice's components: the contraction parts' slots summed in slot
            # order, written to shared memory in groups of four components (one 16-byte vector
            # per group and atom, groups NS vectors apart) at position t + OFF (OFF = 0: the
            # slice alone; OFF = BEGIN: every slice of the atom in one array), component t by the
            # lane with t % TPA == sub of the atom's TPA lanes
            out.append("  template <class T, int TPA, int NS, int OFF = 0> static __device__ __forceinline__ void "
                       "adj_to_shared(const T* __restrict__ sl, T* __restrict__ dst, const int sub) {")
            for t, ci in enumerate(comps):
                terms = [f"sl[{s * 32}]" for s in range(slot_begin[ci], slot_begin[ci + 1])] or ["T(0)"]
                out.append(f"    if ({t} % TPA == sub) dst[(({t} + OFF) / 4) * 4 * NS + ({t} + OFF) % 4] = "
                           + " + ".join(terms) + ";")
                # a compiler fence after every 16 components of this lane: the loads of one group
                # are in flight together, not all of them (their registers would set the kernel's
                # count); with four or more lanes per atom a lane's share is small and needs none
                out.append(f'    if (TPA <= 2 && {t + 1} % (16 * TPA) == 0) asm volatile("" ::: "memory");')
            out.append("  }")
        out += _mom_function(prog, monos, comps)
        # adjoint of one pair: P_mu = sum_m adj[mu,m] m gives the radial part s = sum_mu df_mu P_mu;
        # alpha_m = sum_mu adj[mu,m] f_mu times the gradient of each monomial gives the rest
        grads = set()
        for m in monos:
            for k in range(3):
                if m[k] > 0:
                    mm = list(m)
                    mm[k] -= 1
                    grads.add(tuple(mm))
        need = _closure(set(monos) | grads)
        out.append("  template <class T, class A> static __device__ __forceinline__ void grad(const T x, const T y, "
                   "const T z, const T* __restrict__ f, const T* __restrict__ df, const A adj, "
                   "T& s, T& gx, T& gy, T& gz) {")
        out += ["    " + l for l in _mono_code(need, "T")]
        by_m = defaultdict(list)
        for t, ci in enumerate(comps):
            mu, m = prog.comp_list[ci]
            by_m[m].append((t, mu))
        mus = sorted({mu for ts in by_m.values() for _, mu in ts})
        p_terms = defaultdict(list)
        for m in monos:
            nm = None if m == (0, 0, 0) else _mono_name(m)
            for t, mu in by_m[m]:
                p_terms[mu].append(f"adj[{t}]" if nm is None else f"adj[{t}] * {nm}")
        for mu in mus:
            out.append(f"    const T P{mu} = " + " + ".join(p_terms[mu]) + ";")
        out.append("    s += " + " + ".join(f"df[{mu}] * P{mu}" for mu in mus) + ";")
        if tag == "f" and prog.L >= FOLD_GRAD_MIN_LEVEL:
            out += ["    " + l for l in _grad_terms_folded(monos, by_m)]
        else:
            for m in monos:
                if m == (0, 0, 0):
                    continue
                terms = by_m[m]
                al = " + ".join(f"adj[{t}] * f[{mu}]" for t, mu in terms)
                out.append(f"    {{ const T al = {al};")
                for k, gv in enumerate(("gx", "gy", "gz")):
                    if m[k] > 0:
                        mm = list(m)
                        mm[k] -= 1
                        mm = tuple(mm)
                        src = "T(1)" if mm == (0, 0, 0) else _mono_name(mm)
                        coef = "" if m[k] == 1 else f"T({m[k]}) * "
                        out.append(f"      {gv} += {coef}al * {src};")
                out.append("    }")
        out.append("  }")
        # tangent of the moments along per-pair displacements u (loss gradient):
        #   acc[t] += df[mu] (r-hat . u) mono + f[mu] (grad mono . u)
        out.append("  template <class T> static __device__ __forceinline__ void tmom(const T x, const T y, const T z, "
                   "const T* __restrict__ f, const T* __restrict__ df, const T rdu, const T ux, const T uy, const T uz, "
                   "T* __restrict__ acc) {")
        out += ["    " + l for l in _mono_code(need, "T")]
        for t, ci in enumerate(comps):
            mu, m = prog.comp_list[ci]
            mv = "T(1)" if m == (0, 0, 0) else _mono_name(m)
            gterms = []
            for k, uv in enumerate(("ux", "uy", "uz")):
                if m[k] > 0:
                    mm = list(m)
                    mm[k] -= 1
                    mm = tuple(mm)
                    src = "T(1)" if mm == (0, 0, 0) else _mono_name(mm)
                    coef = "" if m[k] == 1 else f"T({m[k]}) * "
                    gterms.append(f"{coef}{src} * {uv}")
            g = " + ".join(gterms) if gterms else "T(0)"
            out.append(f"    acc[{t}] += df[{mu}] * rdu * {mv} + f[{mu}] * ({g});")
        out.append("  }")
        # P_mu = sum adj mono and its tangent Pd_mu = sum adjt mono + adj (grad mono . u), with the
        # adjoint values read from the tile layout (stride 32) starting at this slice
        out.append("  template <class T> static __device__ __forceinline__ void pdot(const T x, const T y, const T z, "
                   "const T* __restrict__ adjp, const T* __restrict__ adjtp, const T ux, const T uy, const T uz, "
                   "T* __restrict__ P, T* __restrict__ Pd) {")
        out += ["    " + l for l in _mono_code(need, "T")]
        for t, ci in enumerate(comps):
            mu, m = prog.comp_list[ci]
            mv = "T(1)" if m == (0, 0, 0) else _mono_name(m)
            gterms = []
            for k, uv in enumerate(("ux", "uy", "uz")):
                if m[k] > 0:
                    mm = list(m)
                    mm[k] -= 1
                    mm = tuple(mm)
                    src = "T(1)" if mm == (0, 0, 0) else _mono_name(mm)
                    coef = "" if m[k] == 1 else f"T({m[k]}) * "
                    gterms.append(f"{coef}{src} * {uv}")
            g = " + ".join(gterms) if gterms else "T(0)"
            out.append(f"    {{ const T av = adjp[{t * 32}], atv = adjtp[{t * 32}];")
            out.append(f"      P[{mu}] += av * {mv}; Pd[{mu}] += atv * {mv} + av * ({g}); }}")
        out.append("  }")
        out.append("};")
    return out


# ---------------------------------------------------------------------------------------------
# Emission
# ---------------------------------------------------------------------------------------------
SLICE_F32 = int(os.environ.get("MTP_SLICE_F32", "136"))
SLICE_F64 = 64


def flop_counts(prog: Program):
    """Algorithmic floating-point operations of one atom (per pair and per atom parts)."""
    C = len(prog.comp_list)
    monos = {m for _, m in prog.comp_list}
    n_mono = len([m for m in monos if m != (0, 0, 0)])
    n_ops = len(prog.ops)
    return {
        "components": C,
        "monomials": n_mono,
        "program_ops": n_ops,
        # per pair: moments 2C + monomials; adjoint: 4C (P, alpha) + 2 N_mu (s) + 2 per nonzero
        # gradient term + monomials; plus the geometry/radial terms added by the caller
        "pair_moments": 2 * C + n_mono,
        "pair_adjoint": 4 * C + 2 * prog.n_mu + 2 * sum(sum(1 for k in range(3) if m[k] > 0) for m in monos)
        + 2 * n_mono,
        # per atom: forward 2 flops per op, adjoint 4 flops per op (two contributions of 2 flops)
        "atom_program": 2 * n_ops + 4 * n_ops,
    }


# Straight-line thread-per-atom contraction up to this level.  Up to lev_max 16 it fits the register
# file (~900 bytes of spills); at 18-20 ptxas keeps most values in local memory, which is still 5.8x
# faster than the warp-cooperative program at lev_max 20 (measured on a 1M-atom cell).
UNROLLED_MAX_LEVEL = int(os.environ.get("MTP_UNROLLED_MAX_LEVEL", "20"))


# The float contraction is split by basis functions into CONTRACT_PARTS[L] programs; each part evaluates the sub-network its basis functions need (shared
# sub-networks are recomputed by every part that needs them), so that one part's values fit in
# registers.  Each warp runs one part for 32 atoms.
CONTRACT_PARTS = {2: 1, 4: 1, 6: 1, 8: 1, 10: 1, 12: 2, 14: 2, 16: 4, 18: 8, 20: 8}
PART_BALANCE = 0.2  # weight of a part's operation count against its value count when assigning


def partition_program(prog: Program, parts: int, balance: float = PART_BALANCE):
    """Split the basis functions into `parts` groups.  Greedy, largest sub-network first: each
    basis function joins the group whose value set grows least, plus `balance` times the group's
    operation count (so that parts take similar time).  Returns [(values, basis indices)]."""
    by_k = defaultdict(list)
    for (k, i, j, w) in prog.ops:
        by_k[k].append((i, j))
    deps = {}
    for k in sorted(set(range(prog.n_values))):
        d = {k}
        for (i, j) in by_k.get(k, []):
            d |= deps[i]
            d |= deps[j]
        deps[k] = frozenset(d)
    nops = {k: len(v) for k, v in by_k.items()}
    groups = [(set(), []) for _ in range(parts)]
    gops = [0] * parts
    order = sorted(range(len(prog.basis_value)), key=lambda a: (-len(deps[prog.basis_value[a]]), a))
    for a in order:
        d = deps[prog.basis_value[a]]
        best = None
        for g in range(parts):
            new = d - groups[g][0]
            add = sum(nops.get(k, 0) for k in new)
            cost = len(groups[g][0]) + len(new) + balance * (gops[g] + add)
            if best is None or cost < best[0]:
                best = (cost, g, add)
        _, g, add = best
        groups[g][0].update(d)
        groups[g][1].append(a)
        gops[g] += add
    return [(vals, sorted(alphas)) for vals, alphas in groups]


def emit_parts(prog: Program, parts: int):
    """Straight-line float contraction split into parts (see CONTRACT_PARTS).  Part g reads the
    moments it needs from the tile layout (src[c * 32]), computes its values in creation order, its
    share of the site energy and of b, then the adjoint of its sub-network seeded by its own basis
    functions, and writes dV/dM of its moments to adjoint slots (dst[slot * 32]).  Slots are
    numbered by component, then part, so that dV/dM_c is the sum of slots slot_begin[c] ..
    slot_begin[c + 1] - 1 in that order."""
    C = len(prog.comp_list)
    by_k = defaultdict(list)
    for (k, i, j, w) in prog.ops:
        by_k[k].append((i, j, w))
    groups = partition_program(prog, parts)
    slot_of = {}
    slot_begin = []
    for c in range(C):
        slot_begin.append(len(slot_of))
        for g, (vals, _) in enumerate(groups):
            if c in vals:
                slot_of[(g, c)] = len(slot_of)
    slot_begin.append(len(slot_of))
    out = [f"#define MTPGEN_HAS_PARTS 1", f"constexpr int NPART = {parts}, NSLOT = {len(slot_of)};",
           "static __device__ const int slot_begin[] = {" + ",".join(map(str, slot_begin)) + "};",
           "template <int PART> struct Part;"]

    def lit(w):
        return "" if w == 1.0 else f"{w!r}f * "

    for g, (vals, alphas) in enumerate(groups):
        out.append(f"template <> struct Part<{g}> {{")
        out.append("  template <bool WANT_B> static __device__ __forceinline__ float run(const float* __restrict__ src, "
                   "float* __restrict__ dst, const float* __restrict__ xi, double* __restrict__ bout) {")
        comps = sorted(v for v in vals if v < C)
        for c in comps:
            out.append(f"    const float v{c} = src[{c * 32}];")
        inner = sorted(v for v in vals if v >= C)
        for k in inner:
            terms = [f"{lit(w)}v{i} * v{j}" for (i, j, w) in by_k[k]]
            out.append(f"    const float v{k} = " + " + ".join(terms) + ";")
        out.append("    float e = 0.f;")
        seed = defaultdict(list)
        for a in alphas:
            v = prog.basis_value[a]
            out.append(f"    e += xi[{a}] * v{v};")
            out.append(f"    if (WANT_B) bout[{a}] = (double)v{v};")
            seed[v].append(a)
        declared = set()

        def aref(v):
            if v not in declared:
                declared.add(v)
                init = " + ".join(f"xi[{a}]" for a in seed.get(v, [])) or "0.f"
                out.append(f"    float a{v} = {init};")
            return f"a{v}"

        for k in reversed(inner):
            ak = aref(k)
            for (i, j, w) in by_k[k]:
                ai = aref(i)
                aj = aref(j)
                out.append(f"    {ai} += {lit(w)}v{j} * {ak};")
                out.append(f"    {aj} += {lit(w)}v{i} * {ak};")
        for c in comps:
            out.append(f"    dst[{slot_of[(g, c)] * 32}] = {aref(c)};")
        out.append("    return e;")
        out.append("  }")
        out.append("};")
    out.append("template <bool WANT_B>")
    out.append("__device__ __forceinline__ float contract_part(int part, const float* __restrict__ src, "
               "float* __restrict__ dst, const float* __restrict__ xi, double* __restrict__ bout) {")
    out.append("  switch (part) {")
    for g in range(parts):
        out.append(f"    case {g}: return Part<{g}>::template run<WANT_B>(src, dst, xi, bout);")
    out.append("  }")
    out.append("  return 0.f;")
    out.append("}")
    return out


# Parts of the tangent (forward-over-reverse) contraction of the loss gradient: every value carries
# a tangent, so a part holds twice the values of a forward part and wants more parts.
DUAL_PARTS = {2: 1, 4: 1, 6: 1, 8: 1, 10: 1, 12: 2, 14: 4, 16: 8, 18: 16, 20: 16}


def emit_dual_parts(prog: Program, parts: int):
    """Straight-line tangent contraction split into parts, for the loss gradient (Sec. 2.2).  Part g
    reads moments M and their tangents T (directional derivatives along the force and stress
    residuals) for its sub-network, evaluates values v and tangents t (t_k = sum w (t_i v_j + v_i t_j)),
    adds ek v - t of its basis functions over the warp's 32 atoms into dxt[alpha] (lane 0 writes),
    then runs the adjoint a and its tangent at (seeds: xi, 0) and writes dV/dM and its tangent of
    its moments to dual slots (adj[slot * 32], adt[slot * 32]), numbered by component then part."""
    C = len(prog.comp_list)
    by_k = defaultdict(list)
    for (k, i, j, w) in prog.ops:
        by_k[k].append((i, j, w))
    groups = partition_program(prog, parts)
    slot_of = {}
    slot_begin = []
    for c in range(C):
        slot_begin.append(len(slot_of))
        for g, (vals, _) in enumerate(groups):
            if c in vals:
                slot_of[(g, c)] = len(slot_of)
    slot_begin.append(len(slot_of))
    out = [f"constexpr int NDPART = {parts}, NDSLOT = {len(slot_of)};",
           "static __device__ const int dslot_begin[] = {" + ",".join(map(str, slot_begin)) + "};",
           "template <int PART> struct DPart;"]

    def lit(w):
        return "" if w == 1.0 else f"{w!r}f * "

    for g, (vals, alphas) in enumerate(groups):
        out.append(f"template <> struct DPart<{g}> {{")
        out.append("  static __device__ __forceinline__ void run(const float* __restrict__ m, const float* __restrict__ mt, "
                   "float* __restrict__ adj, float* __restrict__ adt, const float* __restrict__ xi, double ek, bool act, "
                   "bool lane0, double* __restrict__ dxt) {")
        comps = sorted(v for v in vals if v < C)
        for c in comps:
            out.append(f"    const float v{c} = m[{c * 32}], t{c} = mt[{c * 32}];")
        inner = sorted(v for v in vals if v >= C)
        for k in inner:
            out.append(f"    const float v{k} = " + " + ".join(f"{lit(w)}v{i} * v{j}" for (i, j, w) in by_k[k]) + ";")
            out.append(f"    const float t{k} = " + " + ".join(f"{lit(w)}(t{i} * v{j} + v{i} * t{j})"
                                                           for (i, j, w) in by_k[k]) + ";")
        seed = defaultdict(list)
        for a in alphas:
            v = prog.basis_value[a]
            seed[v].append(a)
            out.append(f"    {{ double d = act ? ek * (double)v{v} - (double)t{v} : 0.0;")
            out.append("      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);")
            out.append(f"      if (lane0) dxt[{a}] = d; }}")
        declared = set()

        def aref(v):
            if v not in declared:
                declared.add(v)
                init = " + ".join(f"xi[{a}]" for a in seed.get(v, [])) or "0.f"
                out.append(f"    float a{v} = {init}, b{v} = 0.f;")
            return f"a{v}", f"b{v}"

        for k in reversed(inner):
            ak, bk = aref(k)
            for (i, j, w) in by_k[k]:
                ai, bi = aref(i)
                aj, bj = aref(j)
                out.append(f"    {ai} += {lit(w)}v{j} * {ak}; {bi} += {lit(w)}(t{j} * {ak} + v{j} * {bk});")
                out.append(f"    {aj} += {lit(w)}v{i} * {ak}; {bj} += {lit(w)}(t{i} * {ak} + v{i} * {bk});")
        for c in comps:
            a_, b_ = aref(c)
            out.append(f"    adj[{slot_of[(g, c)] * 32}] = {a_}; adt[{slot_of[(g, c)] * 32}] = {b_};")
        out.append("  }")
        out.append("};")
    out.append("__device__ __forceinline__ void dual_part(int part, const float* m, const float* mt, float* adj, float* adt, "
               "const float* xi, double ek, bool act, bool lane0, double* dxt) {")
    out.append("  switch (part) {")
    for g in range(parts):
        out.append(f"    case {g}: DPart<{g}>::run(m, mt, adj, adt, xi, ek, act, lane0, dxt); return;")
    out.append("  }")
    out.append("}")
    return out


def emit_level(L, outdir):
    prog = build_program(L)
    fwd_rows, fwd_layers = encode_layout(forward_layout(prog))
    adj_rows, adj_layers = encode_layout(adjoint_layout(prog))
    C = len(prog.comp_list)
    V = prog.n_values
    assert V < 65535
    table = level_table(prog.basis)
    s32 = slices(prog, SLICE_F32)
    sm32 = moment_slices(prog, SLICE_F32)
    s64 = slices(prog, SLICE_F64)
    fl = flop_counts(prog)
    tag = f"L{L}"
    lines = [f"// Generated by paper_2007_08555_gb300/codegen.py for lev_max = {L}. Do not edit.",
             "#pragma once", "#include \"mtp_gen_common.h\"", f"namespace mtpgen_{tag} {{"]
    lines.append(f"constexpr int L = {L}, C = {C}, V = {V}, M = {prog.basis.m}, NMU = {prog.n_mu}, "
                 f"NUMAX = {prog.numax};")
    lines.append(f"constexpr int NS32 = {len(s32)}, NS64 = {len(s64)}, MAXS32 = {max(len(c) for _, c in s32)}, "
                 f"NSM32 = {len(sm32)};")
    lines.append(f"constexpr int FWD_ROWS = {len(fwd_rows)}, ADJ_ROWS = {len(adj_rows)};")
    lines.append(f"constexpr int FWD_LAYERS = {len(fwd_layers)}, ADJ_LAYERS = {len(adj_layers)};")
    lines.append(f"constexpr int PROGRAM_OPS = {len(prog.ops)};")
    lines.append(f"constexpr int FLOP_PAIR_MOMENTS = {fl['pair_moments']}, FLOP_PAIR_ADJOINT = {fl['pair_adjoint']}, "
                 f"FLOP_ATOM_PROGRAM = {fl['atom_program']};")
    lines.append("static const int level_table[] = {" + ",".join(map(str, table)) + "};")
    lines.append(f"constexpr int LEVEL_TABLE_LEN = {len(table)};")
    lines.append("static const int basis_value[] = {" + ",".join(map(str, prog.basis_value)) + "};")
    lines.append("static const unsigned char comp_mu[] = {" + ",".join(str(mu) for mu, _ in prog.comp_list) + "};")
    lines.append("static const unsigned char comp_abc[] = {" +
                 ",".join(f"{a},{b},{c}" for _, (a, b, c) in prog.comp_list) + "};")

    # one 64-bit word per (row, lane): i | j << 16 | k << 32 | flags << 48 | weight index << 51
    weights = sorted({float(ww) for rows in (fwd_rows, adj_rows) for row in rows for (_, _, _, _, ww) in row})
    widx = {w: k for k, w in enumerate(weights)}
    assert len(weights) < (1 << 13)

    def rows_to_c(name, rows):
        words = []
        for row in rows:
            for (a, b, k, f, ww) in row:
                words.append(f"{a | (b << 16) | (k << 32) | (f << 48) | (widx[float(ww)] << 51)}ull")
        lines.append(f"static const unsigned long long {name}_ops[] = {{" + ",".join(words or ["0ull"]) + "};")

    lines.append(f"constexpr int NWEIGHTS = {len(weights)};")
    lines.append("static const float weights[] = {" + ",".join(repr(w) for w in weights) + "};")
    rows_to_c("fwd", fwd_rows)
    rows_to_c("adj", adj_rows)
    lines.append("static const int fwd_layer_rows[] = {" + ",".join(str(e) for _, e in fwd_layers) + "};")
    lines.append("static const int adj_layer_rows[] = {" + ",".join(str(e) for _, e in adj_layers) + "};")
    # slices
    for name, sl in (("s32", s32), ("s64", s64)):
        lines.append(f"static const int {name}_begin[] = {{" +
                     ",".join(str(min(c)) for _, c in sl) + "};")
        lines.append(f"static const int {name}_size[] = {{" + ",".join(str(len(c)) for _, c in sl) + "};")
        for s, (_, comps) in enumerate(sl):
            assert comps == list(range(min(comps), min(comps) + len(comps)))
    nparts, nslots, has_parts = 1, 0, False
    ndparts, ndslots = 1, 0
    if L <= UNROLLED_MAX_LEVEL and prog.ops:
        has_parts = True
        nparts = CONTRACT_PARTS.get(L, 1)
        part_lines = emit_parts(prog, nparts)
        slot_begin = [int(x) for x in part_lines[2].split("{")[1].rstrip("};").split(",")]
        nslots = int(part_lines[1].split("NSLOT = ")[1].rstrip(";"))
        lines += part_lines
        ndparts = DUAL_PARTS.get(L, nparts)
        dual_lines = emit_dual_parts(prog, ndparts)
        ndslots = int(dual_lines[0].split("NDSLOT = ")[1].rstrip(";"))
        lines += dual_lines
    else:
        lines.append("#define MTPGEN_HAS_PARTS 0")
    lines += emit_slice_functions(prog, s32, "f", slot_begin if has_parts else None)
    lines += emit_slice_functions(prog, s64, "d")
    lines += emit_slice_functions(prog, sm32, "mf")
    lines.append("struct Traits {")
    lines.append("  static constexpr int L_ = L, C_ = C, V_ = V, M_ = M, NMU_ = NMU, NUMAX_ = NUMAX, NS32_ = NS32, NS64_ = NS64, "
                 "MAXS32_ = MAXS32, NSM32_ = NSM32;")
    lines.append(f"  static constexpr int NPART_ = {nparts}, NSLOT_ = {max(nslots, 1)};")
    lines.append(f"  static constexpr bool HAS_PARTS_ = {'true' if has_parts else 'false'};")
    lines.append(f"  static constexpr int NDPART_ = {ndparts}, NDSLOT_ = {max(ndslots, 1)};")
    lines.append("  template <int S> using F32 = SliceF<S>;")
    lines.append("  template <int S> using F64 = SliceD<S>;")
    lines.append("  template <int S> using MF32 = SliceMF<S>;")
    lines.append("};")
    lines.append(f"}}  // namespace mtpgen_{tag}")
    path = os.path.join(outdir, f"mtp_gen_{tag}.h")
    text = "\n".join(lines) + "\n"
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as fh:
            fh.write(text)
    return path, {"C": C, "V": V, "m": prog.basis.m, "ops": len(prog.ops), "fwd_rows": len(fwd_rows),
                  "adj_rows": len(adj_rows), "slices32": len(s32), "slices64": len(s64), **fl}


def emit_tu(L, outdir):
    """One translation unit per level: instantiates the kernels of mtp_level_impl.cuh."""
    text = (f"// Generated by paper_2007_08555_gb300/codegen.py for lev_max = {L}. Do not edit.\n"
            f"#include \"mtp_gen_L{L}.h\"\n"
            f"#define MTP_GEN_NS mtpgen_L{L}\n"
            f"#define MTP_LEVEL_FN mtp_level_ops_L{L}\n"
            f"#include \"mtp_level_impl.cuh\"\n")
    path = os.path.join(outdir, f"mtp_level_L{L}.cu")
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as fh:
            fh.write(text)
    return path


def emit_all(outdir, levels=SUPPORTED_LEVELS):
    os.makedirs(outdir, exist_ok=True)
    info = {}
    for L in levels:
        info[L] = emit_level(L, outdir)[1]
        emit_tu(L, outdir)
    return info


if __name__ == "__main__":
    import sys
    import json

    print(json.dumps(emit_all(sys.argv[1] if len(sys.argv) > 1 else "generated"), indent=1))

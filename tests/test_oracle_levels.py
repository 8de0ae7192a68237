"""Pins of the oracle's basis enumeration (Sec. 2.1, Eqs. 5-6).

* the nine functions of lev_max = 8 listed in Eq. 6 (golden file);
* the level examples printed after Eq. 5 (golden file);
* an independent brute-force enumeration (every edge multiset of every label multiset,
  deduplicated with networkx's labelled-multigraph isomorphism) gives the same set for lev_max <= 12.
"""

import itertools
import os

import networkx as nx
import pytest
from networkx.algorithms.isomorphism import categorical_multiedge_match, categorical_node_match

from oracle import levels

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _sig_component(labels, edges):
    """Isomorphism-invariant signature of a small connected contraction: sorted labels plus
    the sorted multiset of (label_a, label_b, multiplicity) edges."""
    e = sorted(tuple(sorted([labels[i], labels[j]])) + (k,) for (i, j), k in edges.items())
    return (tuple(sorted(labels)), tuple(e))


def _sig_basis(b, lev_max):
    comps = levels.connected_components(lev_max)
    out = []
    for k in b.components:
        c = comps[k]
        a = c.matrix()
        edges = {(i, j): a[i][j] for i in range(c.n) for j in range(i + 1, c.n) if a[i][j]}
        out.append(_sig_component(list(c.labels), edges))
    return tuple(sorted(out))


def _parse_paper_factor(tok):
    tok = tok.strip()
    for sep, mult in ((":", 2), (".", 1)):
        if sep in tok:
            a, b = tok.split(sep)
            la = (int(a[1]), int(a[2]))
            lb = (int(b[1]), int(b[2]))
            return _sig_component([la, lb], {(0, 1): mult})
    return _sig_component([(int(tok[1]), int(tok[2]))], {})


def test_eq6_lev8_basis_matches_paper():
    paper = []
    for line in open(os.path.join(GOLD, "basis_lev8.txt")):
        if line.startswith("#") or not line.strip():
            continue
        lev, expr = line.split("|")
        paper.append((int(lev), tuple(sorted(_parse_paper_factor(t) for t in expr.split("*")))))
    ours = [(b.level, _sig_basis(b, 8)) for b in levels.basis(8)]
    assert len(ours) == 9
    assert sorted(ours) == sorted(paper)


def test_level_examples_after_eq5():
    for line in open(os.path.join(GOLD, "level_examples.txt")):
        if line.startswith("#") or not line.strip():
            continue
        lev, labels, edges = [p.strip() for p in line.split("|")]
        labs = [tuple(int(x) for x in t.split(",")) for t in labels.split()]
        total = sum(levels.moment_level(mu, nu) for mu, nu in labs)
        assert total == int(lev), line
        # the contraction pattern is consistent: every index of every moment is used exactly once
        deg = [0] * len(labs)
        for e in edges.split():
            ij, k = e.split("x")
            i, j = (int(x) for x in ij.split("-"))
            deg[i] += int(k)
            deg[j] += int(k)
        assert deg == [nu for _, nu in labs] or len(labs) == 1 or all(nu == 0 for _, nu in labs)


def _brute_force_basis_signatures(lev_max):
    """Every product of connected contractions with total level <= lev_max, enumerated without the
    oracle's canonical form: all label multisets, all edge multisets, networkx isomorphism."""
    labels_all = [(mu, nu) for mu in range(lev_max) for nu in range(lev_max + 1)
                  if levels.moment_level(mu, nu) <= lev_max]
    comps = []  # (level, graph)
    for n in range(1, lev_max // 2 + 1):
        for labs in itertools.combinations_with_replacement(labels_all, n):
            lev = sum(levels.moment_level(*x) for x in labs)
            if lev > lev_max:
                continue
            if n == 1:
                if labs[0][1] == 0:
                    g = nx.MultiGraph()
                    g.add_node(0, lab=labs[0])
                    comps.append((lev, g))
                continue
            if any(nu == 0 for _, nu in labs):
                continue
            pairs = list(itertools.combinations(range(n), 2))
            maxm = max(nu for _, nu in labs)
            for mult in itertools.product(range(maxm + 1), repeat=len(pairs)):
                deg = [0] * n
                for (i, j), k in zip(pairs, mult):
                    deg[i] += k
                    deg[j] += k
                if deg != [nu for _, nu in labs]:
                    continue
                g = nx.MultiGraph()
                for i, lab in enumerate(labs):
                    g.add_node(i, lab=lab)
                for (i, j), k in zip(pairs, mult):
                    for _ in range(k):
                        g.add_edge(i, j)
                if not nx.is_connected(g):
                    continue
                if any(l2 == lev and nx.is_isomorphic(g, g2, node_match=categorical_node_match("lab", None),
                                                      edge_match=categorical_multiedge_match("x", None))
                       for l2, g2 in comps):
                    continue
                comps.append((lev, g))
    # signatures of components, then products (multisets) of components
    csig = []
    for lev, g in comps:
        labels = [g.nodes[i]["lab"] for i in range(g.number_of_nodes())]
        edges = {}
        for i, j in g.edges():
            key = (min(i, j), max(i, j))
            edges[key] = edges.get(key, 0) + 1
        csig.append((lev, _sig_component(labels, edges)))
    out = set()

    def rec(start, chosen, lev):
        if chosen:
            out.add((lev, tuple(sorted(csig[k][1] for k in chosen))))
        for k in range(start, len(csig)):
            if lev + csig[k][0] <= lev_max:
                rec(k, chosen + [k], lev + csig[k][0])

    rec(0, [], 0)
    return out


@pytest.mark.parametrize("lev_max", [2, 4, 6, 8, 10, 12])
def test_enumeration_matches_independent_brute_force(lev_max):
    ours = {(b.level, _sig_basis(b, lev_max)) for b in levels.basis(lev_max)}
    assert len(ours) == len(levels.basis(lev_max))  # signatures are unique at these sizes
    assert ours == _brute_force_basis_signatures(lev_max)


def test_count_sequence_and_ordering():
    # counts for lev_max = 2..20 (8 -> 9 is the paper's, Eq. 6; the rest follow from the definition
    # and are pinned by the brute-force test up to 12)
    counts = [len(levels.basis(L)) for L in range(2, 21, 2)]
    assert counts == [1, 2, 5, 9, 17, 32, 61, 116, 229, 460]
    for L in (10, 16):
        keys = [(b.level, b.n_moments, b.components) for b in levels.basis(L)]
        assert keys == sorted(keys)
        assert all(b.level % 2 == 0 for b in levels.basis(L))


def test_used_moments_rule():
    # a moment (mu, nu) occurs iff nu = 0 and 2 + 4 mu <= L, or nu >= 1 and 4 mu + 2 nu <= L - 4
    for L in range(2, 21, 2):
        expect = {(mu, nu) for mu in range(L) for nu in range(L)
                  if (nu == 0 and 2 + 4 * mu <= L) or (nu >= 1 and 4 * mu + 2 * nu <= L - 4)}
        assert set(levels.used_moments(L)) == expect

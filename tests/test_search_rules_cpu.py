"""The two rules by which the GPU cluster search prunes (LOOP mode), restated
in plain Python and checked against the oracle's enumerator on random
multigraphs.  (1) Closing level: below a set S of size K - 2, the clusters of
size K are S + U[i] + U[j] with U[j] a later candidate of S joining two
vertices already in S + U[i] and covering its degree-one vertices; no set of
size K - 1 needs to be expanded.  (2) Two-bond closing test: a child of size
K - 2 whose degree-one vertices cannot be served within two more candidate
bonds (cost 1 for a bond to the child, 2 for a path through one outside
vertex, costs summing to <= 4) has no cluster below it.  The GPU kernels
implement the same rules; these tests check the rules, the GPU parity tests
check the kernels."""
import numpy as np
import pytest

from paper_2512_10910_gb300 import inputs as I
from oracle import enumerate as E


def _graph(seed):
    rng = np.random.default_rng(500 + seed)
    n = 5 + seed % 5
    m = n + 3 + seed % 7
    deg = [0] * n
    edges = [(v, v + 1) for v in range(n - 1)]
    for a, b in edges:
        deg[a] += 1; deg[b] += 1
    while len(edges) < m:
        a, b = (int(x) for x in rng.integers(0, n, size=2))
        if a == b or deg[a] >= 6 or deg[b] >= 6:
            continue
        edges.append((min(a, b), max(a, b)))
        deg[a] += 1; deg[b] += 1
    return n, edges


def _search(n, edges, K, closing):
    """Redelmeier search from the smallest bond; LOOP mode; with `closing`,
    the size K - 2 sets are closed directly and their children filtered by
    the two-bond test."""
    inc = [[] for _ in range(n)]
    for e, (a, b) in enumerate(edges):
        inc[a].append(e); inc[b].append(e)
    out = set()

    def other(e, v):
        a, b = edges[e]
        return b if a == v else a

    def deg_of(S):
        d = {}
        for e in S:
            for v in edges[e]:
                d[v] = d.get(v, 0) + 1
        return d

    def dangling(S):
        return [v for v, k in deg_of(S).items() if k == 1]

    def closable2(S, U):
        # S: the child (size K - 2), U: its candidate list
        V = set(deg_of(S))
        D = dangling(S)
        if len(D) > 4:
            return False
        total = 0
        for v in D:
            cost = 3
            for q in U:
                if v not in edges[q]:
                    continue
                w = other(q, v)
                if w in V:
                    cost = 1
                    break
                if any(f != q and w in edges[f] and other(f, w) in V for f in U):
                    cost = min(cost, 2)
            if cost > 2:
                return False
            total += cost
        return total <= 4

    def rec(S, U, anchor):
        V = set(deg_of(S))
        if closing and len(S) == K - 2:
            for i, e in enumerate(U):
                C = S + [e]
                D = dangling(C)
                if not D:
                    out.add(tuple(sorted(C)))
                if len(D) <= 2:
                    Vc = set(deg_of(C))
                    for f in U[i + 1:]:
                        if all(x in Vc for x in edges[f]) and all(d in edges[f] for d in D):
                            out.add(tuple(sorted(C + [f])))
            return
        for i, e in enumerate(U):
            C = S + [e]
            D = dangling(C)
            if not D:
                out.add(tuple(sorted(C)))
            if len(C) >= K or len(D) > 2 * (K - len(C)):
                continue
            new_v = [v for v in edges[e] if v not in V]
            nu = []
            if new_v:
                b = new_v[0]
                nu = [f for f in inc[b] if f != e and f > anchor and other(f, b) not in V and other(f, b) != b]
            Uc = U[i + 1:] + nu
            # every degree-one vertex needs a later candidate touching it
            if any(not any(d in edges[f] for f in Uc) for d in D):
                continue
            if closing and len(C) == K - 2 and not closable2(C, Uc):
                continue
            rec(C, Uc, anchor)

    for a in range(len(edges)):
        x0, x1 = edges[a]
        U = [f for f in inc[x0] if f > a] + [f for f in inc[x1] if f > a and other(f, x1) != x0]
        if K >= 2:
            rec([a], U, a)
    return out


@pytest.mark.parametrize("seed", range(12))
def test_closing_level_and_two_bond_test_keep_every_cluster(seed):
    n, edges = _graph(seed)
    g = I.grid_graph(n, edges, [2] * len(edges))
    for K in (3, 4, 5, 6, 7):
        ref = {tuple(sorted(c)) for c in E.clusters_grow(g, K, E.LOOP)}
        assert _search(n, edges, K, closing=False) == ref, (seed, K)
        assert _search(n, edges, K, closing=True) == ref, (seed, K)

"""Writes tests/golden/cluster_counts.json from the CPU oracle only.

Counts of LOOP clusters by size and of terms by order, for lattices too large
for the oracle to enumerate inside a test run.  Each entry records the oracle
routine that produced it.  Run:  python tests/golden/make_golden.py [name ...]
(no names: every case; named cases are recomputed and merged into the file).

The 8x8x8 lattice at order 10 is counted by the oracle's per-anchor growth
over anchor ranges in parallel worker processes (the ranges are independent
and their counts add up); its terms are the empty term, the clusters, and the
vertex-disjoint pairs, which the minimum cluster size 4 limits to clusters of
size <= 6 (no triple fits in order 10).
"""
import json
import os
import sys
import time
from collections import Counter
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2512_10910_gb300 import inputs as I  # noqa: E402
from oracle import enumerate as E  # noqa: E402

CASES = [
    ("square16x16", lambda: I.square_lattice(16, 16, 2), 8),
    ("square24x24", lambda: I.square_lattice(24, 24, 2), 8),
    ("cubic6x6x6", lambda: I.cubic_lattice(6, 6, 6, 2), 8),
    ("cubic8x8x8", lambda: I.cubic_lattice(8, 8, 8, 2), 8),
    ("cubic4x4x4_K10", lambda: I.cubic_lattice(4, 4, 4, 2), 10),
    ("cubic8x8x8_K10", lambda: I.cubic_lattice(8, 8, 8, 2), 10),
]
PARALLEL = {"cubic8x8x8_K10": (8, 8, 8)}      # lattice dimensions, rebuilt in each worker


def _range_counts(args):
    dims, K, a0, a1 = args
    g = I.cubic_lattice(*dims, 2)
    return E.count_clusters_by_size_range(g, K, E.LOOP, a0, a1, even=True)


def _is_even(g, cluster):
    deg = Counter(int(v) for b in cluster for v in g.bond_site[b])
    return all(d % 2 == 0 for d in deg.values())


def parallel_case(g, K, dims):
    """Clusters by size from anchor ranges counted side by side; terms from the
    clusters and the disjoint pairs of clusters of size <= K - 4.  The same for
    even subgraphs (every vertex of even degree: the terms whose Ising value is
    tanh(beta)^order, all others vanishing), from the even clusters."""
    chunks = [(dims, K, a, min(a + 8, g.n_bonds)) for a in range(0, g.n_bonds, 8)]
    by = [0] * (K + 1)
    ev = [0] * (K + 1)
    with ProcessPoolExecutor(max_workers=max(1, os.cpu_count() - 1), mp_context=mp.get_context("spawn")) as ex:
        for part, epart in ex.map(_range_counts, chunks):
            by = [x + y for x, y in zip(by, part)]
            ev = [x + y for x, y in zip(ev, epart)]
    small = E.clusters_grow(g, K - 4, E.LOOP)                 # sizes 4..K-4
    tuples = E.enumerate_terms(g, small, K)
    assert all(len(tt) <= 2 for tt in tuples)
    pairs = Counter(sum(len(small[i]) for i in tt) for tt in tuples if len(tt) == 2)
    even_pairs = Counter(sum(len(small[i]) for i in tt) for tt in tuples
                         if len(tt) == 2 and all(_is_even(g, small[i]) for i in tt))
    by_size = {k: v for k, v in enumerate(by) if v}
    by_order = Counter(by_size)
    by_order[0] += 1
    for k, v in pairs.items():
        by_order[k] += v
    even_by_order = Counter({k: v for k, v in enumerate(ev) if v})
    even_by_order[0] += 1
    for k, v in even_pairs.items():
        even_by_order[k] += v
    return sum(by), sum(by_order.values()), by_size, by_order, even_by_order


def main(names):
    path = os.path.join(HERE, "cluster_counts.json")
    out = {"generator": "oracle.enumerate.clusters_grow + enumerate_terms (LOOP mode); "
                        "cubic8x8x8_K10: oracle.enumerate.count_clusters_by_size_range over anchor ranges",
           "cases": {}}
    if names and os.path.exists(path):
        out["cases"] = json.load(open(path))["cases"]
    for name, geom, K in CASES:
        if names and name not in names:
            continue
        g = geom()
        t = time.time()
        extra = {}
        if name in PARALLEL:
            n_cl, n_t, by_size, by_order, even = parallel_case(g, K, PARALLEL[name])
            extra = {"even_terms_by_order": {str(k): v for k, v in sorted(even.items())}}
        else:
            cl = E.clusters_grow(g, K, E.LOOP)
            terms = E.enumerate_terms(g, cl, K)
            n_cl, n_t = len(cl), len(terms)
            by_size = Counter(len(c) for c in cl)
            by_order = Counter(sum(len(cl[i]) for i in tt) for tt in terms)
        out["cases"][name] = {"K": K, "n_sites": g.n_sites, "n_bonds": g.n_bonds, "n_clusters": n_cl,
                              "n_terms": n_t, "clusters_by_size": {str(k): v for k, v in sorted(by_size.items())},
                              "terms_by_order": {str(k): v for k, v in sorted(by_order.items())},
                              "seconds": round(time.time() - t, 1), **extra}
        print(name, out["cases"][name], flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])

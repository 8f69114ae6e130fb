"""Writes tests/golden/cluster_counts.json from the CPU oracle only.

Counts of LOOP clusters by size and of terms by order, for lattices too large
for the oracle to enumerate inside a test run.  Each entry records the oracle
routine that produced it.  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys
import time
from collections import Counter

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
]


def main():
    out = {"generator": "oracle.enumerate.clusters_grow + enumerate_terms (LOOP mode)", "cases": {}}
    for name, geom, K in CASES:
        g = geom()
        t = time.time()
        cl = E.clusters_grow(g, K, E.LOOP)
        terms = E.enumerate_terms(g, cl, K)
        by_size = Counter(len(c) for c in cl)
        by_order = Counter(sum(len(cl[i]) for i in tt) for tt in terms)
        out["cases"][name] = {"K": K, "n_sites": g.n_sites, "n_bonds": g.n_bonds, "n_clusters": len(cl),
                              "n_terms": len(terms), "clusters_by_size": {str(k): v for k, v in sorted(by_size.items())},
                              "terms_by_order": {str(k): v for k, v in sorted(by_order.items())},
                              "seconds": round(time.time() - t, 1)}
        print(name, out["cases"][name], flush=True)
    with open(os.path.join(HERE, "cluster_counts.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

"""Multi-index partitions and the combinatorial form of the PNE (oracle; FP64).

Test infrastructure only (see ``oracle/__init__.py``).

* A partition p is a set S_p of closed bonds, drawn as a line transecting those
  indices (Sec. II.C).  Its projector factorises over the transected bonds
  (Eq. A8), each factor the rank-1 projector of the BP fixed point (Eq. A7,
  Eq. A10): P_p = (x)_{b in S_p} P_b.  Its complement Q_p = I - P_p acts on
  all of S_p jointly and does not factorise (Eq. A9).
* Z(o_1, ..., o_M) is the network with operator o_p inserted on the bonds of
  partition p and the identity everywhere else (Sec. II.A notation).  Two
  partitions may transect the same bond; their operators then act one after
  the other along it.  The rank-1 factors commute and P_b P_b = P_b, so
  inserting several P_p amounts to P_b once on every bond of their union, and
  Eq. A6 (inclusion-exclusion over commuting projectors) still holds.
* Combinatorial form (Eq. A6), exact for any complementary P and Q:
      Z0 = Z(Q_1, ..., Q_M) + sum_{x != 0} (-1)^{|x|+1} Z(P^{(x)x}),
  where x runs over the non-empty subsets of the M partitions and P^{(x)x}
  inserts P_p for p in x and the identity on the others.  The approximation
  keeps the 2^M - 1 sub-networks and neglects the residue Z(Q_1, ..., Q_M).
* Linear form (Eq. A4) over partitions: Z0 = Z(Q_1..Q_M) +
  sum_r Z(Q_1, ..., Q_r, P_{r+1}, I, ..., I).
* Every sub-network is contracted here as written, by one einsum over the
  whole network with the operators inserted (small networks only).
"""
from __future__ import annotations

import math
from itertools import combinations

import numpy as np

from . import bp as _bp
from .expansion import _compact_labels, site_values, neumaier

__all__ = ["contract_inserted", "partition_projector", "partition_complement", "comb_subsets",
           "combinatorial_pne", "residue_direct", "linear_pne", "terms_touching_all"]


def contract_inserted(net, inserts) -> float:
    """Z of the closed network with multi-bond operators inserted.  ``inserts``
    is a list of (bonds, op): ``bonds`` a tuple of closed bond ids, ``op`` an
    array of shape [d_b for b in bonds] * 2 whose first half of axes faces the
    first site of each bond (bond_site[b][0]) and second half the second site.
    Operators that share a bond are applied along it in list order (composed:
    the operators of one expansion commute, so the order does not matter);
    bonds in no insert carry the identity."""
    label = {}                       # current label of each bond, walking from s0 to s1
    nxt = [2 * net.n_bonds]

    def fresh():
        nxt[0] += 1
        return nxt[0] - 1
    ops_in = []
    for bonds, op in inserts:
        ins, outs = [], []
        for b in bonds:
            b = int(b)
            if int(net.bond_site[b][1]) < 0:
                raise ValueError("closed networks only")
            ins.append(label.get(b, 2 * b))
            o = fresh()
            outs.append(o)
            label[b] = o
        ops_in.append((np.asarray(op, dtype=np.float64), ins + outs))
    ops = []
    for v in range(net.n_sites):
        labels = []
        for b in net.legs(v):
            b = int(b)
            s0, s1 = int(net.bond_site[b][0]), int(net.bond_site[b][1])
            if s1 < 0:
                raise ValueError("closed networks only")
            labels.append(label.get(b, 2 * b) if s1 == v else 2 * b)
        ops += [np.asarray(net.tensors[v], dtype=np.float64), labels]
    for t, labels in ops_in:
        ops += [t, labels]
    return float(np.einsum(*_compact_labels(ops), [], optimize="greedy"))


def partition_projector(proj, S) -> np.ndarray:
    """P_p = (x)_{b in S} P_b (Eq. A8), axes [s0 sides..., s1 sides...]."""
    out = np.ones(())
    for b in S:
        out = np.multiply.outer(out, proj[b][0])
    n = len(S)
    # outer product axes come as (a0, c0, a1, c1, ...): regroup to (a..., c...)
    return np.transpose(out, [2 * i for i in range(n)] + [2 * i + 1 for i in range(n)])


def partition_complement(proj, S) -> np.ndarray:
    """Q_p = I - P_p on the bonds of S jointly (Eq. A9: not a product)."""
    P = partition_projector(proj, S)
    dims = [P.shape[i] for i in range(len(S))]
    n = int(np.prod(dims))
    return (np.eye(n) - P.reshape(n, n)).reshape(dims + dims)


def comb_subsets(M):
    """The 2^M - 1 non-empty subsets x of the partitions, by size then
    lexicographically, with their sign (-1)^{|x|+1} (Eq. A6)."""
    out = []
    for k in range(1, M + 1):
        for x in combinations(range(M), k):
            out.append((x, 1 if k % 2 == 1 else -1))
    return out


def _bp_projectors(net, tol=1e-13, max_iter=10000):
    r = _bp.bp_fixed_point(net, tol=tol, max_iter=max_iter)
    if not r.converged:
        raise RuntimeError("BP did not converge")
    return _bp.bond_projectors(net, r)


def combinatorial_pne(net, partitions, proj=None):
    """The combinatorial PNE with the residue neglected.  Returns a dict:
    ``terms`` [(x, sign, Z(P^x))], ``c`` per-order sums c_k = sum_{|x|=k}
    Z(P^x) / Z_ref (k = 0..M, c_0 = 0; Z_ref = product of the nonzero site
    values z_v, as in the linear form), ``value`` = sum_k (-1)^{k+1} Z_ref c_k,
    and the projectors used."""
    if proj is None:
        proj = _bp_projectors(net)
    M = len(partitions)
    terms = []
    for x, sign in comb_subsets(M):
        # every active partition's projector; it factorises (Eq. A8), so it
        # is inserted as its single-bond factors P_b (composed where two
        # active partitions share a bond)
        inserts = [((int(b),), proj[int(b)][0]) for p in x for b in partitions[p]]
        terms.append((x, sign, contract_inserted(net, inserts)))
    z = site_values(net, proj)
    nz = z[z != 0.0]
    zref = float(np.prod(nz)) if len(nz) else 1.0
    c = np.zeros(M + 1)
    for k in range(1, M + 1):
        c[k] = neumaier(v / zref for (x, s, v) in terms if len(x) == k)
    value = neumaier(s * v for (x, s, v) in terms)
    return {"terms": terms, "c": c, "value": value, "zref": zref, "proj": proj, "n_terms": len(terms)}


def residue_direct(net, partitions, proj) -> float:
    """Z(Q_1, ..., Q_M): every partition's complement inserted (Eq. res)."""
    inserts = [(tuple(int(b) for b in S), partition_complement(proj, S)) for S in partitions]
    return contract_inserted(net, inserts)


def linear_pne(net, partitions, proj) -> float:
    """The linear form over partitions (Eq. A4), residue neglected:
    sum_{r=0}^{M-1} Z(Q_1, ..., Q_r, P_{r+1}, I, ..., I)."""
    total = []
    for r in range(len(partitions)):
        inserts = [(tuple(int(b) for b in partitions[p]), partition_complement(proj, partitions[p])) for p in range(r)]
        inserts.append((tuple(int(b) for b in partitions[r]), partition_projector(proj, partitions[r])))
        total.append(contract_inserted(net, inserts))
    return neumaier(total)


def terms_touching_all(clusters, terms, partitions):
    """For loop-series terms (tuples of cluster ids): the excited bond set of
    each, and whether it meets every partition (those are the residue's
    terms when the projectors come from a BP fixed point)."""
    sets = [frozenset(int(b) for b in S) for S in partitions]
    out = []
    for t in terms:
        E = set()
        for i in t:
            E.update(int(b) for b in clusters[i])
        out.append((t, len(E), all(E & S for S in sets)))
    return out

"""Recursive partitioning (Sec. IV.A) (oracle; FP64).

Test infrastructure only (see ``oracle/__init__.py``).

* A first set of partitions (chosen for a small residue) gives the
  combinatorial form (Eq. A6): every non-empty subset x contributes
  (-1)^{|x|+1} Z(P^x).  The sub-network of x falls apart along the bonds of
  the partitions in x ("cut" bonds) into connected components.
* A sub-network with a component too costly to contract is not contracted
  as it is but expanded again by the combinatorial form over the
  second-level partitions whose bonds all join sites of such a component and
  none of which is cut.  On a square lattice (site id = y * lx + x) the cost
  of contracting a component grows with the shorter side of its bounding box
  (a strip of width w carries w legs from row to row: O(chi^(2w)) for the
  paper's blocks), so a component is too costly when both sides of its box
  exceed ``max_side``:
      Z(P^x) ~ sum_{y != 0} (-1)^{|y|+1} Z(P^x P^y),
  the second level's residue neglected.  With one too-large component (the
  paper's 4 x 3 example, one 3 x 3 block per sub-network) this is that
  component's own expansion times the values of the others.  A sub-network
  that no second-level partition fits is contracted as it is.
* The projectors are the rank-r projectors of the weighted network (Sec. V.A,
  ``oracle.weights``); every contraction is the whole network with the
  projectors inserted, as written (``oracle.combinatorial``).
"""
from __future__ import annotations

from .combinatorial import comb_subsets, contract_inserted, partition_complement
from .expansion import neumaier

__all__ = ["components", "recursive_combinatorial"]


def components(net, cut):
    """Connected components (lists of sites, ascending) of the graph of the
    closed bonds not in ``cut``."""
    parent = list(range(net.n_sites))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for b in range(net.n_bonds):
        s0, s1 = (int(x) for x in net.bond_site[b])
        if s1 < 0 or b in cut:
            continue
        ra, rb = find(s0), find(s1)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    groups = {}
    for v in range(net.n_sites):
        groups.setdefault(find(v), []).append(v)
    return sorted(groups.values())


def _inserts_p(proj, bonds):
    return [((int(b),), proj[int(b)][0]) for b in sorted(bonds)]


def _too_costly(C, lx, max_side):
    xs = [v % lx for v in C]
    ys = [v // lx for v in C]
    return min(max(xs) - min(xs) + 1, max(ys) - min(ys) + 1) > max_side


def recursive_combinatorial(net, parts1, parts2, proj, lx, max_side, with_residue2=False):
    """The two-level expansion.  Returns a dict: ``value`` (residues of both
    levels neglected; with ``with_residue2`` the second level's residue
    Z(P^x Q_y1 ... Q_yn), complements inserted directly, is added back to each
    expanded sub-network, which makes it exact at the second level),
    ``contractions`` (networks contracted), ``expanded`` (the subsets x that
    were expanded again) and ``levels`` [(x, sign, value)]."""
    total, levels, expanded = [], [], []
    n_contr = 0
    for x, sign in comb_subsets(len(parts1)):
        cut = set(int(b) for p in x for b in parts1[p])
        comps = components(net, cut)
        big = [set(C) for C in comps if _too_costly(C, lx, max_side)]
        sub = []
        if big:
            for S in parts2:
                bs = [int(b) for b in S]
                if any(b in cut for b in bs):
                    continue
                inside = all(any(int(net.bond_site[b][0]) in C and int(net.bond_site[b][1]) in C for C in big)
                             for b in bs)
                if inside:
                    sub.append(bs)
        if not sub:
            val = contract_inserted(net, _inserts_p(proj, cut))
            n_contr += 1
        else:
            expanded.append(x)
            vals = []
            for y, s2 in comb_subsets(len(sub)):
                bonds = set(cut) | set(b for q in y for b in sub[q])
                vals.append(s2 * contract_inserted(net, _inserts_p(proj, bonds)))
                n_contr += 1
            if with_residue2:
                ins = _inserts_p(proj, cut) + [(tuple(S), partition_complement(proj, S)) for S in sub]
                vals.append(contract_inserted(net, ins))
            val = neumaier(vals)
        levels.append((x, sign, val))
        total.append(sign * val)
    return {"value": neumaier(total), "contractions": n_contr, "expanded": expanded, "levels": levels}

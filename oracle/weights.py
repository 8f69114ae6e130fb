"""Weight passing and rank-r projectors (oracle; FP64).

Test infrastructure only (see ``oracle/__init__.py``).

* ``weight_passing`` follows App. C: every closed bond carries a diagonal
  matrix of positive weights S_i, initially the identity.  One update of bond
  i between tensors A and B absorbs the weights of A's other legs into A (A')
  and of B's other legs into B (B'), takes the SVDs A' = U_A S_A V_A^T and
  B' = U_B S_B V_B^T between index i and the rest (Eq. weight1), then the SVD
  S_A V_A^T S_i U_B S_B = U_C S_C V_C^T (Eq. weight2), and replaces
      A -> A V_A S_A^{-1} U_C S_C^{(1-alpha)/2},
      B -> S_C^{(1-alpha)/2} V_C^T S_B^{-1} U_B^T B,
      S_i -> S_C^alpha                                   (Eq. weight3),
  a pure change of gauge: the network with every S_i inserted keeps its
  value.  Sweeps run over the bonds in id order until the weights stop
  changing.  The weights are rescaled to a largest entry of 1 after each
  update, the factor kept in a log scale (the paper is silent on this).
* ``weighted_network`` absorbs sqrt(S_i) into both ends of every bond: a plain
  network with the same value, in which the rank-r projector onto the r
  largest weights of bond i (Sec. V.A) is diagonal: the first r index values
  (the SVD orders S_C descending).
* ``rank_r_linear`` / ``rank_r_combinatorial``: the linear form (Eq. A4) and
  the combinatorial form (Eq. A6) over partitions with those projectors,
  every sub-network contracted as written (``oracle.combinatorial``).
"""
from __future__ import annotations

import math

import numpy as np

from .combinatorial import contract_inserted, comb_subsets, partition_complement, partition_projector
from .expansion import neumaier

__all__ = ["weight_passing", "weighted_network", "rank_r_projectors", "rank_r_linear", "rank_r_combinatorial"]


def _leg_pos(net, v, b):
    legs = [int(x) for x in net.legs(v)]
    return legs.index(int(b))


def _absorb_others(net, tensors, S, v, skip):
    """Tensor of site v with the weight of every leg except bond ``skip``
    multiplied in (full weight, A' of App. C)."""
    t = np.asarray(tensors[v], dtype=np.float64)
    for i, b in enumerate(int(x) for x in net.legs(v)):
        if b == skip:
            continue
        shape = [1] * t.ndim
        shape[i] = -1
        t = t * S[b].reshape(shape)
    return t


def _as_matrix(t, pos):
    """Matrix [rest, leg pos] with the remaining legs in order."""
    t = np.moveaxis(t, pos, -1)
    return t.reshape(-1, t.shape[-1]), t.shape


def weight_passing(net, alpha=0.8, tol=1e-12, max_sweeps=5000):
    """Returns (tensors, S, log_scale, sweeps, change): the network with S_b
    inserted on every closed bond, times exp(log_scale), has the value of the
    input network."""
    tensors = [np.asarray(t, dtype=np.float64).copy() for t in net.tensors]
    S = [np.ones(int(net.bond_dim[b])) for b in range(net.n_bonds)]
    log_scale = 0.0
    change = math.inf
    for sweep in range(1, max_sweeps + 1):
        change = 0.0
        for b in range(net.n_bonds):
            u, v = int(net.bond_site[b][0]), int(net.bond_site[b][1])
            if v < 0:
                continue
            pa, pb = _leg_pos(net, u, b), _leg_pos(net, v, b)
            Am, _ = _as_matrix(_absorb_others(net, tensors, S, u, b), pa)          # [rest_A, d]
            Bm, _ = _as_matrix(_absorb_others(net, tensors, S, v, b), pb)          # [rest_B, d]
            # A' = U_A S_A V_A^T over (rest, i); B' = U_B S_B V_B^T over (i, rest)
            _, sa, vat = np.linalg.svd(Am, full_matrices=False)                 # vat: V_A^T [k, d]
            ubt, sb, _ = np.linalg.svd(Bm.T, full_matrices=False)               # ubt: U_B [d, k]
            if len(sa) != len(S[b]) or len(sb) != len(S[b]):
                raise ValueError("weight passing needs every bond dimension <= the rest of its tensors")
            Mx = (sa[:, None] * vat) @ (S[b][:, None] * ubt) * sb[None, :]
            uc, sc, vct = np.linalg.svd(Mx)
            left = vat.T @ np.diag(1.0 / sa) @ uc @ np.diag(sc ** ((1 - alpha) / 2))     # d x d, on A's leg
            right = np.diag(sc ** ((1 - alpha) / 2)) @ vct @ np.diag(1.0 / sb) @ ubt.T   # d x d, on B's leg
            tensors[u] = np.moveaxis(np.tensordot(tensors[u], left, axes=([pa], [0])), -1, pa)
            tensors[v] = np.moveaxis(np.tensordot(right, tensors[v], axes=([1], [pb])), 0, pb)
            new = sc ** alpha
            top = float(new.max())
            log_scale += math.log(top)
            new = new / top
            change = max(change, float(np.max(np.abs(new - S[b]))))
            S[b] = new
        if change < tol:
            return tensors, S, log_scale, sweep, change
    return tensors, S, log_scale, max_sweeps, change


def weighted_network(net, tensors, S, log_scale):
    """sqrt(S_b) absorbed into both ends of every bond; returns (network,
    log_scale): the network's value times exp(log_scale) is the original's."""
    out = []
    for v in range(net.n_sites):
        t = np.asarray(tensors[v], dtype=np.float64)
        for i, b in enumerate(int(x) for x in net.legs(v)):
            shape = [1] * t.ndim
            shape[i] = -1
            t = t * np.sqrt(S[b]).reshape(shape)
        out.append(t)
    return net.with_tensors(out), log_scale


def rank_r_projectors(net, r):
    """Per closed bond: (P, Q, cap0, cap1) with P the diagonal projector onto
    the first r index values (the r largest weights), Q = I - P.  Caps are not
    defined for r > 1 (None)."""
    out = []
    for b in range(net.n_bonds):
        d = int(net.bond_dim[b])
        P = np.diag([1.0 if a < r else 0.0 for a in range(d)])
        out.append((P, np.eye(d) - P, None, None))
    return out


def rank_r_linear(net, partitions, proj):
    """Linear form over partitions (Eq. A4), residue neglected."""
    total = []
    for k in range(len(partitions)):
        inserts = [(tuple(int(b) for b in partitions[p]), partition_complement(proj, partitions[p])) for p in range(k)]
        inserts += [((int(b),), proj[int(b)][0]) for b in partitions[k]]
        total.append(contract_inserted(net, inserts))
    return neumaier(total)


def rank_r_combinatorial(net, partitions, proj):
    """Combinatorial form over partitions (Eq. A6), residue neglected."""
    terms = []
    for x, sign in comb_subsets(len(partitions)):
        inserts = [((int(b),), proj[int(b)][0]) for p in x for b in partitions[p]]
        terms.append(sign * contract_inserted(net, inserts))
    return neumaier(terms)

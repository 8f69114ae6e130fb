"""Belief-propagation messages and rank-1 bond projectors (oracle; FP64).

Test infrastructure only (see ``oracle/__init__.py``).

* ``bp_fixed_point`` -- message passing to a fixed point (Sec. I and
  Sec. II.B: BP messages; Sec. III.D: boundary reflection on open indices).
  Schedule (the paper is silent): Jacobi sweeps from the uniform message
  ``1/sqrt(d)``; each new message is normalised to unit 2-norm and its sign
  fixed so that the entry of largest magnitude (first such index) is positive;
  stop when the largest entry change is below ``tol``.
* ``bond_projectors`` -- rank-1 projector of Eq. A7.  With the two messages
  normalised so that their overlap is one (App. B), ``P_b`` caps each side of
  the cut bond with the message arriving from the other side, and
  ``Q_b = I - P_b`` (Sec. II.A, Fig. 1a).
"""
from __future__ import annotations

import numpy as np

__all__ = ["BPResult", "bp_fixed_point", "bond_projectors", "incoming_slot"]


class BPResult:
    def __init__(self, out, iters, residual, converged):
        self.out = out            # list over leg slots k: outgoing message of the site along leg k
        self.iters = iters
        self.residual = residual
        self.converged = converged


def _slot_table(net):
    """slot[(v, b)] -> position k in ``site_bonds`` of site v's leg on bond b."""
    slot = {}
    for v in range(net.n_sites):
        for k in range(net.site_ptr[v], net.site_ptr[v + 1]):
            slot[(v, int(net.site_bonds[k]))] = k
    return slot


def incoming_slot(net, slot, v, b):
    """Leg slot whose outgoing message arrives at site v along bond b.
    Open index: boundary reflection, the site's own outgoing message (Sec. III.D)."""
    s0, s1 = int(net.bond_site[b][0]), int(net.bond_site[b][1])
    if s1 < 0:
        return slot[(v, b)]
    other = s1 if s0 == v else s0
    return slot[(other, b)]


def _normalise(m):
    nrm = float(np.sqrt(np.dot(m, m)))
    if not nrm > 0.0:
        raise FloatingPointError("zero BP message")
    m = m / nrm
    if m[int(np.argmax(np.abs(m)))] < 0:
        m = -m
    return m


def _site_messages(t, ins):
    """All outgoing messages of one site: for each leg j, contract the site
    tensor with the incoming messages on every other leg."""
    outs = []
    k = t.ndim
    for j in range(k):
        r = t
        for i in reversed(range(k)):        # highest axis first keeps indices valid
            if i == j:
                continue
            r = np.tensordot(r, ins[i], axes=([i], [0]))
        outs.append(np.asarray(r, dtype=np.float64).reshape(-1))
    return outs


def bp_fixed_point(net, tol=1e-13, max_iter=10000, damping=0.0):
    slot = _slot_table(net)
    nslots = len(net.site_bonds)
    out = [np.full(int(net.bond_dim[net.site_bonds[k]]),
                   1.0 / np.sqrt(float(net.bond_dim[net.site_bonds[k]])))
           for k in range(nslots)]
    # incoming slot for every (site, leg)
    inc = [[incoming_slot(net, slot, v, int(b)) for b in net.legs(v)]
           for v in range(net.n_sites)]
    residual = np.inf
    for it in range(1, max_iter + 1):
        new = [None] * nslots
        for v in range(net.n_sites):
            ins = [out[k] for k in inc[v]]
            msgs = _site_messages(net.tensors[v], ins)
            for j, m in enumerate(msgs):
                k = net.site_ptr[v] + j
                if damping > 0.0:
                    m = (1.0 - damping) * _normalise(m) + damping * out[k]
                new[k] = _normalise(m)
        residual = max(float(np.max(np.abs(new[k] - out[k]))) for k in range(nslots)) if nslots else 0.0
        out = new
        if residual < tol:
            return BPResult(out, it, residual, True)
    return BPResult(out, max_iter, residual, False)


def bond_projectors(net, bp: BPResult, degenerate=1e-300):
    """For each closed bond b = (s0, s1): (P_b, Q_b, cap0, cap1) where P_b is a
    matrix [index at s0, index at s1], cap0 is the vector that caps s0's leg
    when the bond is cut (the message arriving at s0), and cap1 = message
    arriving at s1 divided by the overlap n_b, so that P_b = cap0 (x) cap1 and
    P_b @ P_b = P_b.  Open bonds are not partitioned and map to None."""
    slot = _slot_table(net)
    res = []
    for b in range(net.n_bonds):
        s0, s1 = int(net.bond_site[b][0]), int(net.bond_site[b][1])
        if s1 < 0:
            res.append(None)
            continue
        m0 = bp.out[slot[(s0, b)]]       # s0 -> b
        m1 = bp.out[slot[(s1, b)]]       # s1 -> b
        n = float(np.dot(m0, m1))
        if abs(n) < degenerate:
            raise ZeroDivisionError(f"degenerate message overlap on bond {b}")
        cap0 = m1.copy()                 # arrives at s0
        cap1 = m0 / n                    # arrives at s1, carries 1/n_b
        P = np.outer(cap0, cap1)
        Q = np.eye(P.shape[0]) - P
        res.append((P, Q, cap0, cap1))
    return res

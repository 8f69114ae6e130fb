"""Exact references (oracle; FP64).

Test infrastructure only (see ``oracle/__init__.py``).

* ``contract_einsum`` -- Eq. A1 written out: the whole network in one einsum
  (open indices become the output axes in ascending bond id), tiny networks.
* ``contract_sweep`` -- the same contraction site by site in id order,
  carrying the open-frontier tensor and a log scale (lattices up to the width
  where D^(width+1) fits in memory).
* ``ising_spin_sum`` -- the Ising partition function by its definition, a sum
  over every spin configuration (App. A encodes it as a network).
* ``ising_ht`` -- the textbook high-temperature form
  Z = 2^N cosh(bJ)^M sum_k n_k tanh(bJ)^k, n_k = number of even bond subsets.
* ``onsager_minus_beta_f`` -- Onsager's bulk free energy of the square-lattice
  Ising model (-beta f per site), by 2-D quadrature.
* ``relative_error`` / ``eps2`` -- Eq. B1 and Eq. B2.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["contract_einsum", "contract_sweep", "ising_spin_sum", "ising_ht",
           "onsager_minus_beta_f", "relative_error", "eps2", "corner_estimator"]


def contract_einsum(net):
    ops = []
    for v in range(net.n_sites):
        ops += [np.asarray(net.tensors[v], dtype=np.float64), [int(b) for b in net.legs(v)]]
    out = [int(b) for b in net.open_bonds()]
    if net.n_bonds > 52:
        raise ValueError("too many bonds for np.einsum")
    return np.einsum(*ops, out, optimize="greedy")


def contract_sweep(net, order=None):
    """Returns (tensor, log_scale) with the exact result = tensor * exp(log_scale).
    For a closed network the tensor is a 0-d array."""
    order = range(net.n_sites) if order is None else order
    cur = np.ones(())
    labels = []                 # bond id of each axis of cur
    log_scale = 0.0
    open_set = set(int(b) for b in net.open_bonds())
    for v in order:
        t = np.asarray(net.tensors[v], dtype=np.float64)
        legs = [int(b) for b in net.legs(v)]
        shared = [b for b in legs if b in labels]
        ax_cur = [labels.index(b) for b in shared]
        ax_t = [legs.index(b) for b in shared]
        cur = np.tensordot(cur, t, axes=(ax_cur, ax_t))
        labels = [b for b in labels if b not in shared] + [b for b in legs if b not in shared]
        m = float(np.max(np.abs(cur))) if cur.size else 0.0
        if m > 0:
            e = math.floor(math.log2(m))
            cur = cur * 2.0 ** (-e)
            log_scale += e * math.log(2.0)
    # only open bonds remain
    assert set(labels) == open_set, (labels, open_set)
    perm = sorted(range(len(labels)), key=lambda i: labels[i])
    return np.transpose(cur, perm), log_scale


def ising_spin_sum(net, beta, J=1.0):
    """Z = sum over s in {+1,-1}^N of exp(beta J sum_{closed bonds} s_i s_j)."""
    n = net.n_sites
    if n > 24:
        raise ValueError("too many spins")
    idx = np.arange(2 ** n, dtype=np.int64)
    spins = 1 - 2 * ((idx[:, None] >> np.arange(n)) & 1)          # [2^n, n]
    energy = np.zeros(2 ** n)
    for (a, b) in net.bond_site:
        if b >= 0:
            energy += spins[:, a] * spins[:, b]
    e0 = beta * J * energy
    mx = float(np.max(e0))
    return math.exp(mx) * float(np.sum(np.exp(e0 - mx)))


def ising_ht(n_sites, n_bonds, beta, counts, J=1.0):
    """High-temperature expansion value from the even-subgraph counts."""
    t = math.tanh(beta * J)
    s = sum(float(c) * t ** k for k, c in enumerate(counts))
    return (2.0 ** n_sites) * math.cosh(beta * J) ** n_bonds * s


def onsager_minus_beta_f(beta, J=1.0):
    """-beta f = ln 2 + (1/(8 pi^2)) int_0^{2pi} int_0^{2pi}
    ln[cosh^2(2bJ) - sinh(2bJ)(cos t1 + cos t2)] dt1 dt2  (Onsager 1944)."""
    from scipy import integrate
    c2 = math.cosh(2 * beta * J) ** 2
    s2 = math.sinh(2 * beta * J)
    val, _ = integrate.dblquad(lambda t2, t1: math.log(c2 - s2 * (math.cos(t1) + math.cos(t2))),
                               0.0, 2 * math.pi, 0.0, 2 * math.pi, epsabs=1e-13, epsrel=1e-13)
    return math.log(2.0) + val / (8 * math.pi ** 2)


def corner_estimator(lnz_LL, lnz_LLm1, lnz_Lm1Lm1):
    """ln Z(L,L) - 2 ln Z(L,L-1) + ln Z(L-1,L-1): cancels the edge and corner
    terms of an open lattice and leaves the bulk per-site value."""
    return lnz_LL - 2.0 * lnz_LLm1 + lnz_Lm1Lm1


def relative_error(z_exact, z_approx):
    """Eq. B1."""
    return abs((z_exact - z_approx) / z_exact)


def eps2(t_exact, t_approx):
    """Eq. B2: 2-norm error of an open-network tensor."""
    return float(np.linalg.norm(np.ravel(t_exact - t_approx)) / np.linalg.norm(np.ravel(t_exact)))

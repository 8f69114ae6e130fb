"""Term values and the truncated partitioned expansion (oracle; FP64).

Test infrastructure only (see ``oracle/__init__.py``).

Everything here works in the ORIGINAL basis of the site tensors, with the
explicit projector matrices of Eq. A7 and Q = I - P (Sec. II.A, Fig. 1a):

* A term (a P/Q string, Eq. A2-A4) is the network with Q on the bonds of E
  and P on every other bond.  A P bond is cut and each side capped by the
  message arriving from the other side (Sec. II.C).  The term therefore
  factorises into the isolated sites (each fully capped, value ``z_v``) and
  one contraction per connected component C of E, in which C's bonds carry
  explicit Q matrices and every other leg of C's sites is capped (``Z'_C``).
* ``w(C) = Z'_C / prod_{v in C, z_v != 0} z_v`` and ``nz(C)`` = number of sites of
  C with ``z_v == 0``.  A term divided by ``Z_ref = prod_{z_v != 0} z_v`` is
  ``prod_C w(C)`` when its clusters cover every zero site, else 0.
* ``c_k`` = sum over terms of order k of ``Term / Z_ref``, Neumaier-compensated,
  in canonical term order; ``Z_K = Z_ref * sum_{k<=K} c_k``.  Neglecting the
  terms above order K is the truncation of Sec. II.B (the residue and the
  high-degree terms are dropped).
* ``log_series`` (not in the paper; the reading of the non-extensive literal
  sum): ``log|Z_ref| + sum_{k=1..K} [x^k] log(sum_j c_j x^j)``.
"""
from __future__ import annotations

import math
from itertools import product

import numpy as np

from . import bp as _bp
from .enumerate import (LOOP, ALL, enumerate_clusters, enumerate_terms, all_subsets,
                        components, cluster_vertices)

__all__ = ["capped_tensor", "site_values", "cluster_value", "term_value_unfactorized",
           "neumaier", "power_series_log", "pne", "pne_open", "PNEResult"]


def neumaier(values) -> float:
    """Neumaier's compensated sum, in the given order."""
    s = 0.0
    c = 0.0
    for x in values:
        x = float(x)
        t = s + x
        if abs(s) >= abs(x):
            c += (s - t) + x
        else:
            c += (x - t) + s
        s = t
    return s + c


def _compact_labels(ops):
    """np.einsum's sublist form takes labels below 52: renumber them densely."""
    m = {}
    out = []
    for i in range(0, len(ops), 2):
        out.append(ops[i])
        out.append([m.setdefault(x, len(m)) for x in ops[i + 1]])
    if len(m) > 52:
        raise ValueError("too many indices for np.einsum")
    return out


def capped_tensor(net, proj, v, keep=()):
    """Site tensor of v with every closed leg NOT in ``keep`` capped by the
    message arriving along it (Sec. II.C: cut and capped).  Remaining axes
    follow the ascending bond ids in ``keep``."""
    t = np.asarray(net.tensors[v], dtype=np.float64)
    legs = [int(b) for b in net.legs(v)]
    for i in reversed(range(len(legs))):
        b = legs[i]
        if b in keep:
            continue
        if proj[b] is None:
            raise ValueError("open legs must be sliced before the expansion")
        _, _, cap0, cap1 = proj[b]
        cap = cap0 if int(net.bond_site[b][0]) == v else cap1
        t = np.tensordot(t, cap, axes=([i], [0]))
    return t


def site_values(net, proj) -> np.ndarray:
    """z_v: each site capped on all legs (the all-P term's site factors)."""
    return np.array([float(capped_tensor(net, proj, v)) for v in range(net.n_sites)])


def cluster_value(net, proj, C) -> float:
    """Z'_C: contraction of C's sites (capped off C) with explicit Q_b on C's bonds."""
    Cset = set(int(b) for b in C)
    verts = cluster_vertices(net, C)
    ops = []
    for v in verts:
        keep = sorted(b for b in (int(x) for x in net.legs(v)) if b in Cset)
        t = capped_tensor(net, proj, v, keep=Cset)
        # label of (bond b, side of v): 2*b + side
        labels = [2 * b + (0 if int(net.bond_site[b][0]) == v else 1) for b in keep]
        ops += [t, labels]
    for b in sorted(Cset):
        ops += [proj[b][1], [2 * b, 2 * b + 1]]
    return float(np.einsum(*_compact_labels(ops), [], optimize="greedy"))


def term_value_unfactorized(net, proj, E) -> float:
    """Term(E) by contracting the whole network with Q on E and P elsewhere,
    no factorisation (tiny networks only)."""
    Eset = set(int(b) for b in E)
    ops = []
    for v in range(net.n_sites):
        labels = [2 * int(b) + (0 if int(net.bond_site[b][0]) == v else 1) for b in net.legs(v)]
        ops += [np.asarray(net.tensors[v], dtype=np.float64), labels]
    for b in range(net.n_bonds):
        P, Q, _, _ = proj[b]
        ops += [Q if b in Eset else P, [2 * b, 2 * b + 1]]
    return float(np.einsum(*_compact_labels(ops), [], optimize="greedy"))


def power_series_log(c, K) -> np.ndarray:
    """l_k = [x^k] log(sum_j c_j x^j) for k = 1..K, with c_0 = 1 (c is divided by
    c_0 first).  Recurrence from f' = f (log f)':
    k l_k = k c_k - sum_{j=1}^{k-1} j l_j c_{k-j}."""
    c = np.asarray(c, dtype=np.float64) / float(c[0])
    l = np.zeros(K + 1)
    with np.errstate(over="ignore", invalid="ignore"):
        _ps_log_fill(c, l, K)
    return l


def _ps_log_fill(c, l, K):
    for k in range(1, K + 1):
        acc = k * (c[k] if k < len(c) else 0.0)
        for j in range(1, k):
            acc -= j * l[j] * (c[k - j] if k - j < len(c) else 0.0)
        l[k] = acc / k


class PNEResult(dict):
    __getattr__ = dict.__getitem__


def _expand(net, proj, K, mode, clusters=None, terms=None):
    z = site_values(net, proj)
    zero = (z == 0.0)
    n_zero = int(np.sum(zero))
    nz_log = float(np.sum(np.log(np.abs(z[~zero])))) if np.any(~zero) else 0.0
    nz_sign = int(np.prod(np.sign(z[~zero]))) if np.any(~zero) else 1
    if mode == ALL and terms is None:
        # every subset of the bonds is a term (small networks only)
        subsets = all_subsets(net, K)
        cache = {}
        rows = []
        for E in subsets:
            val, cover = 1.0, 0
            for C in components(net, E):
                if C not in cache:
                    zc = cluster_value(net, proj, C)
                    vs = cluster_vertices(net, C)
                    den = float(np.prod([z[v] for v in vs if z[v] != 0.0])) if vs else 1.0
                    cache[C] = (zc / den, sum(1 for v in vs if z[v] == 0.0))
                w, nzc = cache[C]
                val *= w
                cover += nzc
            rows.append((len(E), val if cover == n_zero else 0.0))
        n_clusters = len(cache)
        n_terms = len(subsets)
        cl_list, w_list = sorted(cache, key=lambda t: (len(t), t)), None
    else:
        if clusters is None:
            clusters = enumerate_clusters(net, K, mode)
        w_arr = np.empty(len(clusters))
        nz_arr = np.empty(len(clusters), dtype=np.int64)
        for i, C in enumerate(clusters):
            zc = cluster_value(net, proj, C)
            vs = cluster_vertices(net, C)
            den = float(np.prod([z[v] for v in vs if z[v] != 0.0]))
            w_arr[i] = zc / den
            nz_arr[i] = sum(1 for v in vs if z[v] == 0.0)
        if terms is None:
            terms = enumerate_terms(net, clusters, K)
        rows = []
        for t in terms:
            order = sum(len(clusters[i]) for i in t)
            cover = sum(int(nz_arr[i]) for i in t)
            val = float(np.prod([w_arr[i] for i in t])) if t else 1.0
            rows.append((order, val if cover == n_zero else 0.0))
        n_clusters, n_terms = len(clusters), len(terms)
        cl_list, w_list = clusters, w_arr
    c = np.zeros(K + 1)
    a = np.zeros(K + 1)
    for k in range(K + 1):
        vals = [v for (o, v) in rows if o == k]
        c[k] = neumaier(vals)
        a[k] = neumaier(abs(v) for v in vals)
    total = neumaier(c)
    sign = nz_sign * (1 if total >= 0 else -1)
    log_abs = nz_log + (math.log(abs(total)) if total != 0 else -math.inf)
    if n_zero == 0 and c[0] != 0:
        l = power_series_log(c, K)
        log_series = nz_log + float(np.sum(l[1:])) + math.log(abs(c[0]))
    else:
        log_series = math.nan
    return PNEResult(z=z, n_zero=n_zero, log_abs_zref=nz_log, sign_zref=nz_sign,
                     c=c, abs_c=a, sum_c=total, sign=sign, log_abs=log_abs,
                     value=sign * math.exp(log_abs) if log_abs < 700 else sign * math.inf,
                     log_series=log_series, n_clusters=n_clusters, n_terms=n_terms,
                     clusters=cl_list, w=w_list, terms=terms)


def pne(net, K, mode=LOOP, tol=1e-13, max_iter=10000, damping=0.0, proj=None,
        clusters=None, terms=None):
    """The truncated PNE of a closed network: BP (Sec. II.B) -> rank-1
    projectors (Eq. A7) -> all terms of order <= K (Eq. A4, residue and higher
    orders dropped) -> per-order sums.  ``proj`` may be supplied (any
    complementary P, Q: the identities of Eq. A2-A4 hold for any choice)."""
    bpres = None
    if proj is None:
        bpres = _bp.bp_fixed_point(net, tol=tol, max_iter=max_iter, damping=damping)
        if not bpres.converged:
            raise RuntimeError("BP did not converge")
        proj = _bp.bond_projectors(net, bpres)
    r = _expand(net, proj, K, mode, clusters=clusters, terms=terms)
    r["bp"] = bpres
    r["proj"] = proj
    return r


def pne_open(net, K, mode=LOOP, tol=1e-13, max_iter=10000):
    """Open-index output (Sec. III.D): BP with boundary reflection on the open
    indices, projectors on the closed bonds only, then one closed network per
    assignment of the open indices (each site tensor sliced), all sharing the
    projectors and the cluster/term lists.  Returns the FP64 tensor over the
    open indices in ascending bond-id order, plus per-entry results."""
    from paper_2512_10910_gb300.inputs import slice_open
    bpres = _bp.bp_fixed_point(net, tol=tol, max_iter=max_iter)
    if not bpres.converged:
        raise RuntimeError("BP did not converge")
    proj_full = _bp.bond_projectors(net, bpres)
    ob = [int(b) for b in net.open_bonds()]
    keep = [b for b in range(net.n_bonds) if b not in set(ob)]
    proj = [proj_full[b] for b in keep]
    dims = [int(net.bond_dim[b]) for b in ob]
    out = np.zeros(dims)
    clusters = terms = None
    entries = {}
    for o in product(*[range(d) for d in dims]):
        sl = slice_open(net, o)
        if clusters is None:
            clusters = enumerate_clusters(sl, K, mode) if mode == LOOP else None
            terms = enumerate_terms(sl, clusters, K) if mode == LOOP else None
        r = _expand(sl, proj, K, mode, clusters=clusters, terms=terms)
        out[o] = r.sign * math.exp(r.log_abs) if r.sum_c != 0 else 0.0
        entries[o] = r
    return out, entries, bpres

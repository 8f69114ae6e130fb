"""Cluster and term enumeration (oracle).

Test infrastructure only (see ``oracle/__init__.py``).

Definitions (Sec. II.A, Eq. A4; Sec. III.A):
* A *term* of the linear expansion with every bond partitioned is a P/Q
  string, i.e. the set E of bonds that carry Q ("excited").  Its order is |E|,
  the number of excited indices (the paper's "degree").
* E splits into connected components ("clusters"), which are pairwise
  vertex-disjoint.  In LOOP mode every cluster is free of dangling excitations
  (no vertex of cluster degree one, Sec. III.A); ALL mode keeps every cluster.
* Canonical order: clusters by (size, sorted bond tuple); terms as increasing
  tuples of canonical cluster ids, in lexicographic order, the empty term first.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from bisect import bisect_right
from itertools import combinations

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "enum_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle_enum.so")
_lib = None

LOOP, ALL = 0, 1


def build_oracle_lib(force=False) -> str:
    """Compile the C part of the oracle with gcc (no GPU involved)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _get_lib():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle_lib())
        p32 = ctypes.POINTER(ctypes.c_int32)
        p64 = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_enum_bitmask.restype = ctypes.c_int64
        lib.oracle_enum_bitmask.argtypes = [ctypes.c_int32, ctypes.c_int32, p32, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32, p32, ctypes.c_int64]
        lib.oracle_enum_grow.restype = ctypes.c_int64
        lib.oracle_enum_grow.argtypes = [ctypes.c_int32, ctypes.c_int32, p32, p32, p32,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, p32,
                                         ctypes.c_int64]
        lib.oracle_count_grow_range.restype = ctypes.c_int32
        lib.oracle_count_grow_range.argtypes = [ctypes.c_int32, ctypes.c_int32, p32, p32, p32, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, p64, p64]
        lib.oracle_even_subsets_by_size.restype = ctypes.c_int32
        lib.oracle_even_subsets_by_size.argtypes = [ctypes.c_int32, ctypes.c_int32, p32, p64]
        _lib = lib
    return _lib


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _canonical(rows: np.ndarray) -> list:
    """rows [n, width] padded with -1 -> list of tuples in canonical order."""
    out = [tuple(int(x) for x in r if x >= 0) for r in rows]
    out.sort(key=lambda t: (len(t), t))
    return out


def clusters_bitmask(net, K, mode=LOOP) -> list:
    """Every subset of the closed bonds tested directly (at most 30 closed bonds)."""
    lib = _get_lib()
    bs = np.ascontiguousarray(net.bond_site, dtype=np.int32)
    width = max(1, min(K, net.n_bonds))
    n = lib.oracle_enum_bitmask(net.n_sites, net.n_bonds, _p32(bs), K, mode, width, None, 0)
    if n < 0:
        raise ValueError("bitmask scan needs <= 30 closed bonds and <= 64 sites")
    out = np.empty((max(n, 1), width), dtype=np.int32)
    lib.oracle_enum_bitmask(net.n_sites, net.n_bonds, _p32(bs), K, mode, width, _p32(out), n)
    return _canonical(out[:n])


def count_clusters_bitmask(net, K, mode=LOOP) -> int:
    """Number of clusters by the bitmask scan, without listing them."""
    lib = _get_lib()
    bs = np.ascontiguousarray(net.bond_site, dtype=np.int32)
    n = lib.oracle_enum_bitmask(net.n_sites, net.n_bonds, _p32(bs), K, mode, max(1, K), None, 0)
    if n < 0:
        raise ValueError("bitmask scan needs <= 30 closed bonds and <= 64 sites")
    return int(n)


def count_clusters_grow(net, K, mode=LOOP) -> int:
    """Number of clusters by per-anchor growth, without listing them."""
    lib = _get_lib()
    bs = np.ascontiguousarray(net.bond_site, dtype=np.int32)
    sp = np.ascontiguousarray(net.site_ptr, dtype=np.int32)
    sb = np.ascontiguousarray(net.site_bonds, dtype=np.int32)
    n = lib.oracle_enum_grow(net.n_sites, net.n_bonds, _p32(bs), _p32(sp), _p32(sb), K, mode, max(1, K), None, 0)
    if n < 0:
        raise MemoryError("oracle_enum_grow failed")
    return int(n)


def count_clusters_by_size_range(net, K, mode, a0, a1, even=False):
    """Clusters by size (index 0..K) whose smallest bond is in [a0, a1), by
    the same per-anchor growth; ranges are independent and add up.  With
    even=True also returns the counts of those clusters whose every vertex has
    even degree (connected even subgraphs)."""
    lib = _get_lib()
    bs = np.ascontiguousarray(net.bond_site, dtype=np.int32)
    sp = np.ascontiguousarray(net.site_ptr, dtype=np.int32)
    sb = np.ascontiguousarray(net.site_bonds, dtype=np.int32)
    by = np.zeros(K + 1, dtype=np.int64)
    ev = np.zeros(K + 1, dtype=np.int64)
    p64 = ctypes.POINTER(ctypes.c_int64)
    st = lib.oracle_count_grow_range(net.n_sites, net.n_bonds, _p32(bs), _p32(sp), _p32(sb), K, mode, a0, a1,
                                     by.ctypes.data_as(p64), ev.ctypes.data_as(p64) if even else None)
    if st != 0:
        raise MemoryError("oracle_count_grow_range failed")
    if even:
        return [int(x) for x in by], [int(x) for x in ev]
    return [int(x) for x in by]


def clusters_grow(net, K, mode=LOOP) -> list:
    """Per-anchor level growth with sort/unique de-duplication (any size)."""
    lib = _get_lib()
    bs = np.ascontiguousarray(net.bond_site, dtype=np.int32)
    sp = np.ascontiguousarray(net.site_ptr, dtype=np.int32)
    sb = np.ascontiguousarray(net.site_bonds, dtype=np.int32)
    width = max(1, K)
    args = (net.n_sites, net.n_bonds, _p32(bs), _p32(sp), _p32(sb), K, mode, width)
    n = lib.oracle_enum_grow(*args, None, 0)
    if n < 0:
        raise MemoryError("oracle_enum_grow failed")
    out = np.empty((max(n, 1), width), dtype=np.int32)
    lib.oracle_enum_grow(*args, _p32(out), n)
    return _canonical(out[:n])


def clusters_python(net, K, mode=LOOP) -> list:
    """Literal definition in pure Python, for tiny networks (<= ~16 closed bonds)."""
    closed = [b for b in range(net.n_bonds) if net.bond_site[b][1] >= 0]
    res = []
    for k in range(1, min(K, len(closed)) + 1):
        for E in combinations(closed, k):
            deg = {}
            for b in E:
                for x in net.bond_site[b]:
                    deg[int(x)] = deg.get(int(x), 0) + 1
            if mode == LOOP and any(d == 1 for d in deg.values()):
                continue
            # connectivity by repeated absorption
            seen = set(int(x) for x in net.bond_site[E[0]])
            left = list(E[1:])
            changed = True
            while changed and left:
                changed = False
                for b in list(left):
                    u, v = int(net.bond_site[b][0]), int(net.bond_site[b][1])
                    if u in seen or v in seen:
                        seen.update((u, v)); left.remove(b); changed = True
            if not left:
                res.append(tuple(E))
    res.sort(key=lambda t: (len(t), t))
    return res


def enumerate_clusters(net, K, mode=LOOP) -> list:
    """Canonical cluster list; bitmask scan when it applies, growth otherwise."""
    if K < 1:
        return []
    n_closed = int(np.sum(net.bond_site[:, 1] >= 0))
    if n_closed <= 30 and net.n_sites <= 64 and (n_closed <= 22 or mode == ALL or K >= n_closed - 4):
        return clusters_bitmask(net, K, mode)
    return clusters_grow(net, K, mode)


def even_subsets_by_size(net) -> np.ndarray:
    """Counts, by size, of bond subsets in which every vertex has even degree."""
    lib = _get_lib()
    bs = np.ascontiguousarray(net.bond_site, dtype=np.int32)
    nc = int(np.sum(net.bond_site[:, 1] >= 0))
    counts = np.zeros(nc + 1, dtype=np.int64)
    r = lib.oracle_even_subsets_by_size(net.n_sites, net.n_bonds, _p32(bs),
                                        counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if r < 0:
        raise ValueError("needs <= 34 closed bonds and <= 64 sites")
    return counts


def cluster_vertices(net, C) -> tuple:
    return tuple(sorted({int(x) for b in C for x in net.bond_site[b]}))


def enumerate_terms(net, clusters, K) -> list:
    """All terms with |E| <= K as increasing tuples of cluster ids whose
    clusters are pairwise vertex-disjoint (Eq. A4: one term per P/Q string;
    its connected components are the clusters).  Lexicographic order, the empty
    term first."""
    sizes = [len(c) for c in clusters]
    vmask = []
    for c in clusters:
        m = 0
        for x in cluster_vertices(net, c):
            m |= 1 << x
        vmask.append(m)
    by_size = {}
    for i, s in enumerate(sizes):
        by_size.setdefault(s, []).append(i)
    size_keys = sorted(by_size)
    out = [()]

    def extend(prefix, used, budget, last):
        # candidates: every cluster id > last whose size fits the budget
        for s in size_keys:
            if s > budget:
                break
            lst = by_size[s]
            for j in lst[bisect_right(lst, last):]:
                if vmask[j] & used:
                    continue
                t = prefix + (j,)
                out.append(t)
                extend(t, used | vmask[j], budget - sizes[j], j)

    extend((), 0, K, -1)
    out.sort()
    return out


def all_subsets(net, K) -> list:
    """ALL mode with full freedom: every subset E of closed bonds, |E| <= K,
    as sorted bond tuples in (size, lexicographic) order."""
    closed = [b for b in range(net.n_bonds) if net.bond_site[b][1] >= 0]
    res = []
    for k in range(0, min(K, len(closed)) + 1):
        res.extend(combinations(closed, k))
    return res


def components(net, E) -> list:
    """Connected components of a bond set (as sorted bond tuples)."""
    E = list(E)
    comps = []
    while E:
        comp = [E.pop(0)]
        verts = set(int(x) for x in net.bond_site[comp[0]])
        changed = True
        while changed:
            changed = False
            for b in list(E):
                u, v = int(net.bond_site[b][0]), int(net.bond_site[b][1])
                if u in verts or v in verts:
                    comp.append(b); verts.update((u, v)); E.remove(b); changed = True
        comps.append(tuple(sorted(comp)))
    return comps

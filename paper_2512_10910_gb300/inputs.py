"""Seeded synthetic inputs: network geometries and site tensors.

This module builds the *problem* (a closed or open tensor network, App. A of the
paper) and holds none of the expansion's arithmetic: no message passing, no
projectors, no cluster or term logic.  Both the CUDA path (through the Python
binding) and the CPU oracle take their inputs from here.

Conventions
-----------
* Sites are numbered ``0..N-1``; bonds ``0..M-1``.
* ``bond_site[b] = (s0, s1)``; ``s1 == -1`` marks an open (dangling) index.
* Each site's legs are its bonds in ascending bond id; ``site_bonds`` is the
  CSR list (``site_ptr``) of those bond ids.
* A site tensor is a float64 C-order array whose axes follow the site's legs.

Tensor recipes (App. A; readings stated in the design notes):
* Ising: sqrt-Boltzmann encoding, ``T_v[a..] = sum_s prod_legs sqrtW[s, a]``
  with ``W[s, s'] = exp(beta J s s')`` (App. A, "Ising Tensors").
* Random: i.i.d. entries from a SplitMix64 stream (App. A, "Random Tensors").
* AKLT: double-layer norm network of the spin-2 square-lattice AKLT PEPS with
  virtual dimension 2 (App. A, "AKLT Tensors").
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Network", "square_lattice", "cubic_lattice", "grid_graph", "with_open_legs",
    "splitmix64_uniform", "splitmix64_normal",
    "ising_tensors", "random_tensors", "aklt_tensors", "slice_open", "batched_workload",
    "uniform_ising", "uniform_random", "uniform_product", "square_lines", "square_block_partitions", "unique_partitions",
]

# leg direction tags stored beside ``site_bonds`` (used by the AKLT builder)
DIR_NONE, DIR_MX, DIR_PX, DIR_MY, DIR_PY, DIR_MZ, DIR_PZ = -1, 0, 1, 2, 3, 4, 5


@dataclass
class Network:
    """Geometry plus (optionally) one set of site tensors."""

    n_sites: int
    bond_site: np.ndarray            # int32 [M, 2]
    bond_dim: np.ndarray             # int32 [M]
    site_ptr: np.ndarray             # int32 [N + 1]
    site_bonds: np.ndarray           # int32 [sum deg]
    leg_dir: np.ndarray              # int8  [sum deg] direction tags (lattices)
    tensors: list = field(default_factory=list)   # list of float64 arrays
    name: str = ""

    @property
    def n_bonds(self) -> int:
        return int(self.bond_site.shape[0])

    def legs(self, v: int) -> np.ndarray:
        return self.site_bonds[self.site_ptr[v]:self.site_ptr[v + 1]]

    def leg_dims(self, v: int) -> tuple:
        return tuple(int(self.bond_dim[b]) for b in self.legs(v))

    def open_bonds(self) -> np.ndarray:
        return np.nonzero(self.bond_site[:, 1] < 0)[0].astype(np.int32)

    def with_tensors(self, tensors, name=None) -> "Network":
        return Network(self.n_sites, self.bond_site, self.bond_dim, self.site_ptr,
                       self.site_bonds, self.leg_dir, list(tensors),
                       self.name if name is None else name)

    def flat_data(self):
        """(data float64 [sum sizes], data_off int64 [N+1]) in site order."""
        sizes = [int(np.prod(self.leg_dims(v))) for v in range(self.n_sites)]
        off = np.zeros(self.n_sites + 1, dtype=np.int64)
        off[1:] = np.cumsum(sizes)
        data = np.empty(int(off[-1]), dtype=np.float64)
        for v in range(self.n_sites):
            t = np.ascontiguousarray(self.tensors[v], dtype=np.float64).reshape(-1)
            assert t.size == sizes[v]
            data[off[v]:off[v + 1]] = t
        return data, off

    def geometry_key(self) -> tuple:
        return (self.n_sites, self.bond_site.tobytes(), self.bond_dim.tobytes())


def _from_bond_list(n_sites, bonds, dims, dirs) -> Network:
    """bonds: list of (s0, s1); dirs: list of (dir at s0, dir at s1)."""
    bond_site = np.asarray(bonds, dtype=np.int32).reshape(-1, 2)
    bond_dim = np.asarray(dims, dtype=np.int32).reshape(-1)
    per_site = [[] for _ in range(n_sites)]
    for b, (s0, s1) in enumerate(bond_site):
        per_site[s0].append((b, dirs[b][0]))
        if s1 >= 0:
            per_site[s1].append((b, dirs[b][1]))
    site_ptr = np.zeros(n_sites + 1, dtype=np.int32)
    sb, sd = [], []
    for v in range(n_sites):
        lst = sorted(per_site[v])
        sb.extend(b for b, _ in lst)
        sd.extend(d for _, d in lst)
        site_ptr[v + 1] = len(sb)
    return Network(n_sites, bond_site, bond_dim, site_ptr,
                   np.asarray(sb, dtype=np.int32), np.asarray(sd, dtype=np.int8))


def square_lattice(lx: int, ly: int, d: int) -> Network:
    """Open-boundary lx-by-ly square lattice; site id = y*lx + x.
    Bonds are numbered site by site: the +x bond, then the +y bond."""
    bonds, dirs = [], []
    for y in range(ly):
        for x in range(lx):
            s = y * lx + x
            if x + 1 < lx:
                bonds.append((s, s + 1)); dirs.append((DIR_PX, DIR_MX))
            if y + 1 < ly:
                bonds.append((s, s + lx)); dirs.append((DIR_PY, DIR_MY))
    net = _from_bond_list(lx * ly, bonds, [d] * len(bonds), dirs)
    net.name = f"square{lx}x{ly}_D{d}"
    return net


def cubic_lattice(lx: int, ly: int, lz: int, d: int) -> Network:
    """Open-boundary cubic lattice; site id = (z*ly + y)*lx + x; bonds numbered
    site by site in the order +x, +y, +z."""
    bonds, dirs = [], []
    for z in range(lz):
        for y in range(ly):
            for x in range(lx):
                s = (z * ly + y) * lx + x
                if x + 1 < lx:
                    bonds.append((s, s + 1)); dirs.append((DIR_PX, DIR_MX))
                if y + 1 < ly:
                    bonds.append((s, s + lx)); dirs.append((DIR_PY, DIR_MY))
                if z + 1 < lz:
                    bonds.append((s, s + lx * ly)); dirs.append((DIR_PZ, DIR_MZ))
    net = _from_bond_list(lx * ly * lz, bonds, [d] * len(bonds), dirs)
    net.name = f"cubic{lx}x{ly}x{lz}_D{d}"
    return net


def grid_graph(n_sites: int, edges, dims) -> Network:
    """Arbitrary geometry from an edge list [(s0, s1), ...] (s1 = -1: open)."""
    return _from_bond_list(n_sites, list(edges), list(dims),
                           [(DIR_NONE, DIR_NONE)] * len(edges))


def with_open_legs(net: Network, legs) -> Network:
    """Append open indices: ``legs`` = [(site, dim), ...].  The new bonds get
    the next bond ids, so each becomes the site's last leg."""
    bonds = [tuple(int(x) for x in b) for b in net.bond_site]
    dims = [int(x) for x in net.bond_dim]
    # recover per-bond direction tags
    dirs = [[DIR_NONE, DIR_NONE] for _ in bonds]
    for v in range(net.n_sites):
        for k in range(net.site_ptr[v], net.site_ptr[v + 1]):
            b = int(net.site_bonds[k])
            side = 0 if net.bond_site[b][0] == v else 1
            dirs[b][side] = int(net.leg_dir[k])
    for s, d in legs:
        bonds.append((int(s), -1)); dims.append(int(d)); dirs.append([DIR_NONE, DIR_NONE])
    out = _from_bond_list(net.n_sites, bonds, dims, [tuple(x) for x in dirs])
    out.name = net.name + f"_open{len(legs)}"
    return out


# ---------------------------------------------------------------------------
# SplitMix64 (Steele, Lea & Flood 2014; constants as published by Vigna)
# ---------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _splitmix64(seed: int, n: int) -> np.ndarray:
    with np.errstate(over="ignore"):
        idx = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1): (x >> 11) * 2^-53 of successive SplitMix64 outputs."""
    return (_splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def splitmix64_normal(seed: int, n: int, mean=0.0, sd=1.0) -> np.ndarray:
    """n normals by Box-Muller (cosine branch), two uniforms per sample."""
    u = splitmix64_uniform(seed, 2 * n)
    u1 = 1.0 - u[0::2]                     # (0, 1]
    u2 = u[1::2]
    return mean + sd * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ---------------------------------------------------------------------------
# Tensor recipes
# ---------------------------------------------------------------------------
def ising_sqrt_boltzmann(beta: float, J: float = 1.0) -> np.ndarray:
    """Symmetric square root of W = [[e^{bJ}, e^{-bJ}], [e^{-bJ}, e^{bJ}]]
    from its eigendecomposition (eigenvectors (1,+-1)/sqrt2)."""
    lp = math.sqrt(2.0 * math.cosh(beta * J))
    lm2 = 2.0 * math.sinh(beta * J)
    if lm2 < 0:
        raise ValueError("antiferromagnetic J needs a complex square root")
    lm = math.sqrt(lm2)
    a, b = 0.5 * (lp + lm), 0.5 * (lp - lm)
    return np.array([[a, b], [b, a]], dtype=np.float64)


def ising_tensors(net: Network, beta: float, J: float = 1.0) -> Network:
    """sqrt-Boltzmann site tensors (bond dim 2); open legs get the same leg
    weight, so they index the spin through sqrtW."""
    sw = ising_sqrt_boltzmann(beta, J)
    tensors = []
    for v in range(net.n_sites):
        k = len(net.legs(v))
        assert all(d == 2 for d in net.leg_dims(v)), "Ising tensors need D=2"
        t = np.zeros((2,) * k)
        for s in range(2):
            term = np.ones(())
            for _ in range(k):
                term = np.multiply.outer(term, sw[s])
            t = t + term
        tensors.append(t)
    return net.with_tensors(tensors, name=net.name + f"_ising_b{beta:g}")


def random_tensors(net: Network, seed: int, dist: str = "u01+0.1") -> Network:
    """Entries from one SplitMix64 stream per network, sites filled in id
    order, each tensor row-major.  dist:
      'u01+0.1'   U[0,1) + 0.1
      'n1,0.3'    N(1, 0.3^2)
      'bias:B'    U[-1+B, 1+B]   (the paper's bias form)."""
    sizes = [int(np.prod(net.leg_dims(v))) for v in range(net.n_sites)]
    n = int(sum(sizes))
    if dist == "u01+0.1":
        vals = splitmix64_uniform(seed, n) + 0.1
    elif dist == "n1,0.3":
        vals = splitmix64_normal(seed, n, 1.0, 0.3)
    elif dist.startswith("bias:"):
        bb = float(dist[5:])
        vals = (2.0 * splitmix64_uniform(seed, n) - 1.0) + bb
    else:
        raise ValueError(dist)
    tensors, p = [], 0
    for v in range(net.n_sites):
        tensors.append(vals[p:p + sizes[v]].reshape(net.leg_dims(v)).copy())
        p += sizes[v]
    return net.with_tensors(tensors, name=net.name + f"_rand{dist}_s{seed}")


def _aklt_single_layer() -> np.ndarray:
    """A[k, l_mx, l_px, l_my, l_py]: spin-2 state k from four spin-1/2 virtual
    legs (symmetric subspace), singlet eps = [[0,1],[-1,0]] applied on the +x
    and +y legs."""
    a = np.zeros((5, 2, 2, 2, 2))
    for bits in range(16):
        idx = [(bits >> (3 - i)) & 1 for i in range(4)]
        k = sum(idx)
        a[(k,) + tuple(idx)] = 1.0 / math.sqrt(math.comb(4, k))
    eps = np.array([[0.0, 1.0], [-1.0, 0.0]])
    a = np.einsum("kabcd,be->kaecd", a, eps)
    a = np.einsum("kabcd,de->kabce", a, eps)
    return a


def aklt_tensors(net: Network) -> Network:
    """Double-layer AKLT norm tensors E = sum_k A^k (x) A^k on a square lattice
    (bond dim 4 = 2x2, ket index major).  Virtual legs with no bond (the
    lattice boundary) are traced between ket and bra."""
    a = _aklt_single_layer()
    # E[(a,a'),(b,b'),...] over the four directions mx, px, my, py
    e = np.einsum("kabcd,kefgh->aebfcgdh", a, a).reshape(4, 4, 4, 4)
    trace_cap = np.eye(2).reshape(4)
    tensors = []
    for v in range(net.n_sites):
        dirs = [int(x) for x in net.leg_dir[net.site_ptr[v]:net.site_ptr[v + 1]]]
        assert all(d in (DIR_MX, DIR_PX, DIR_MY, DIR_PY) for d in dirs)
        assert all(dd == 4 for dd in net.leg_dims(v)), "AKLT norm needs D=4"
        t = e
        # cap missing directions, from the last axis down so indices stay valid
        for dr in (DIR_PY, DIR_MY, DIR_PX, DIR_MX):
            if dr not in dirs:
                t = np.tensordot(t, trace_cap, axes=([dr], [0])) if t.ndim > dr else t
        # remaining axes are in direction order; reorder to the site's leg order
        present = sorted(d for d in (DIR_MX, DIR_PX, DIR_MY, DIR_PY) if d in dirs)
        perm = [present.index(d) for d in dirs]
        tensors.append(np.ascontiguousarray(np.transpose(t, perm)))
    return net.with_tensors(tensors, name=net.name + "_aklt")


def batched_workload_items(indices, n: int = 4096, seed: int = 1234):
    """Only the listed items of batched_workload(n, seed), built the same way
    (the same draws), without building the others."""
    u = splitmix64_uniform(seed, 4 * n).reshape(n, 4)
    out = []
    for i in indices:
        L = 6 + min(18, int(u[i, 0] * 19))
        D = 2 + min(4, int(u[i, 1] * 5))
        if u[i, 2] < 0.5:
            out.append(("random", L, D, None, random_tensors(square_lattice(L, L, D), seed + 1 + i)))
        else:
            beta = 0.3 + 0.2 * float(u[i, 3])
            out.append(("ising", L, 2, beta, ising_tensors(square_lattice(L, L, 2), beta)))
    return out


def batched_workload(n: int = 4096, seed: int = 1234):
    """The uneven batch: n independent open L x L square-lattice networks,
    L uniform in 6..24 and D uniform in 2..6; with probability 1/2 a network is
    random U[0,1)+0.1 at that D, otherwise Ising at D=2 with beta uniform in
    [0.3, 0.5].  Drawn from one SplitMix64 stream; network i's tensors use
    seed + 1 + i.  Returns a list of (kind, L, D, beta or None, Network)."""
    u = splitmix64_uniform(seed, 4 * n).reshape(n, 4)
    out = []
    for i in range(n):
        L = 6 + min(18, int(u[i, 0] * 19))
        D = 2 + min(4, int(u[i, 1] * 5))
        if u[i, 2] < 0.5:
            g = square_lattice(L, L, D)
            out.append(("random", L, D, None, random_tensors(g, seed + 1 + i)))
        else:
            beta = 0.3 + 0.2 * float(u[i, 3])
            g = square_lattice(L, L, 2)
            out.append(("ising", L, 2, beta, ising_tensors(g, beta)))
    return out


def slice_open(net: Network, assignment) -> Network:
    """Fix every open index to a value: returns the closed network obtained by
    slicing each site tensor on its open legs (``assignment`` follows the
    ascending id order of the open bonds)."""
    ob = [int(b) for b in net.open_bonds()]
    val = {b: int(a) for b, a in zip(ob, assignment)}
    keep = [b for b in range(net.n_bonds) if b not in val]
    remap = {b: i for i, b in enumerate(keep)}
    bonds = [tuple(int(x) for x in net.bond_site[b]) for b in keep]
    dims = [int(net.bond_dim[b]) for b in keep]
    tensors = []
    for v in range(net.n_sites):
        t = net.tensors[v]
        legs = [int(b) for b in net.legs(v)]
        sl = tuple(val[b] if b in val else slice(None) for b in legs)
        tensors.append(np.ascontiguousarray(t[sl]))
    dirs = [(DIR_NONE, DIR_NONE)] * len(bonds)
    out = _from_bond_list(net.n_sites, bonds, dims, dirs)
    # legs keep ascending order because remapping is monotone
    del remap
    return out.with_tensors(tensors, name=net.name + "_slice")


# ---------------------------------------------------------------------------
# Partitions (sets of bonds transected by one line) for multi-index PNE
# ---------------------------------------------------------------------------
def bond_between(net: Network, s0: int, s1: int) -> int:
    """Id of the bond joining sites s0 and s1 (either order)."""
    for b in range(net.n_bonds):
        a, c = int(net.bond_site[b][0]), int(net.bond_site[b][1])
        if {a, c} == {s0, s1}:
            return b
    raise KeyError((s0, s1))


def square_line_x(lx: int, ly: int, k: int) -> list:
    """Bonds of an lx-by-ly square lattice crossed by the line between columns
    x = k and x = k + 1 (its +x bonds from column k)."""
    net = square_lattice(lx, ly, 2)
    return sorted(bond_between(net, y * lx + k, y * lx + k + 1) for y in range(ly))


def square_line_y(lx: int, ly: int, k: int) -> list:
    """Bonds crossed by the line between rows y = k and y = k + 1."""
    net = square_lattice(lx, ly, 2)
    return sorted(bond_between(net, k * lx + x, (k + 1) * lx + x) for x in range(lx))


def square_line_diag(lx: int, ly: int, k: int) -> list:
    """Bonds crossed by the anti-diagonal line between the site layers
    x + y = k and x + y = k + 1."""
    net = square_lattice(lx, ly, 2)
    out = []
    for b in range(net.n_bonds):
        u, v = (int(s) for s in net.bond_site[b])
        lu, lv = u % lx + u // lx, v % lx + v // lx
        if sorted((lu, lv)) == [k, k + 1]:
            out.append(b)
    return sorted(out)


def cubic_axis_bonds(l: int, axis: int) -> list:
    """All bonds of an l x l x l cubic lattice along one axis (0: x, 1: y, 2: z)."""
    net = cubic_lattice(l, l, l, 2)
    step = (1, l, l * l)[axis]
    return sorted(b for b in range(net.n_bonds)
                  if abs(int(net.bond_site[b][1]) - int(net.bond_site[b][0])) == step)


def double_loop_vertical() -> list:
    """The double-loop network of six tensors (a 3 x 2 square lattice, two
    plaquettes sharing a bond): its three vertical bonds, one single-index
    partition each."""
    return [[b] for b in square_line_y(3, 2, 0)]


def square3x3_pinwheel() -> list:
    """Four single-index partitions of the 3 x 3 network on boundary bonds, one
    per side, turning the same way around the centre."""
    net = square_lattice(3, 3, 2)
    s = lambda x, y: y * 3 + x
    pairs = [(s(0, 0), s(1, 0)), (s(2, 0), s(2, 1)), (s(0, 1), s(0, 2)), (s(1, 2), s(2, 2))]
    return [[bond_between(net, a, c)] for a, c in pairs]


def square3x3_six_lines() -> list:
    """Six multi-index partitions of the 3 x 3 network: the two vertical and
    the two horizontal lines between rows and columns, the line around the
    corner site 0, and the anti-diagonal line between site layers 1 and 2."""
    return [square_line_x(3, 3, 0), square_line_x(3, 3, 1), square_line_y(3, 3, 0), square_line_y(3, 3, 1),
            square_line_diag(3, 3, 0), square_line_diag(3, 3, 1)]


def cube2_planes() -> list:
    """Three multi-index partitions of the 2 x 2 x 2 network, each the four
    bonds along one axis (cutting one separates two 2 x 2 planes)."""
    return [cubic_axis_bonds(2, a) for a in range(3)]


def ising_blocked(lx: int, ly: int, block: int, beta: float, J: float = 1.0) -> Network:
    """The 2D Ising network of a (lx*block) x (ly*block) open lattice,
    coarse-grained into an lx x ly network: each site is a block x block patch
    of spins contracted over its internal bonds, and the block fine bonds
    crossing between two patches are grouped into one index of dimension
    2^block (row-major over the fine bonds in ascending fine id).  The
    network contracts to the same partition function."""
    fine = ising_tensors(square_lattice(lx * block, ly * block, 2), beta, J)
    FX = lx * block
    coarse = square_lattice(lx, ly, 2 ** block)
    cell = lambda s: ((s % FX) // block, (s // FX) // block)
    # fine bonds crossing each coarse bond
    groups = {b: [] for b in range(coarse.n_bonds)}
    for fb in range(fine.n_bonds):
        u, v = (int(x) for x in fine.bond_site[fb])
        cu, cv = cell(u), cell(v)
        if cu != cv:
            cb = bond_between(coarse, cu[1] * lx + cu[0], cv[1] * lx + cv[0])
            groups[cb].append(fb)
    tensors = []
    for Y in range(ly):
        for X in range(lx):
            c = Y * lx + X
            sites = [s for s in range(fine.n_sites) if cell(s) == (X, Y)]
            lab = {}
            ops = []
            for s in sites:
                ops += [fine.tensors[s], [lab.setdefault(int(b), len(lab)) for b in fine.legs(s)]]
            out = [lab[fb] for cb in coarse.legs(c) for fb in sorted(groups[int(cb)])]
            t = np.einsum(*ops, out, optimize="greedy")
            tensors.append(np.ascontiguousarray(t.reshape(coarse.leg_dims(c))))
    return coarse.with_tensors(tensors, name=f"ising{lx * block}x{ly * block}_blocked{block}_b{beta:g}")


# ---- uniform tensors of infinite square lattices (Sec. IV.C) ----------------
#
# One tensor A repeated on every site of the infinite square lattice, axes
# [l, u, r, d]: l joins the site to its neighbour at x - 1, u to y - 1, r to
# x + 1 and d to y + 1.  A horizontal bond joins the r leg of one site to the l
# leg of the next; a vertical bond the d leg of one site to the u leg of the
# site below.

def uniform_ising(beta: float, block: int = 1, J: float = 1.0) -> np.ndarray:
    """The 2D Ising uniform tensor after a block x block coarse-graining (App.
    A): the block x block patch of sqrt-Boltzmann spin tensors contracted over
    its internal bonds; each leg groups the block fine bonds leaving one side
    (l and r ordered by fine row, u and d by fine column, the first most
    significant), so a leg has dimension 2^block.  One tensor per block^2
    spins: ln Z per tensor is block^2 times ln Z per spin."""
    sw = ising_sqrt_boltzmann(beta, J)
    spin = np.einsum("sa,sb,sc,sd->abcd", sw, sw, sw, sw)
    lab = {}

    def h(x, y):            # bond label right of spin (x, y); x = -1 is the l leg
        return lab.setdefault(("h", x, y), len(lab))

    def v(x, y):            # bond label below spin (x, y); y = -1 is the u leg
        return lab.setdefault(("v", x, y), len(lab))
    ops = []
    for y in range(block):
        for x in range(block):
            ops += [spin, [h(x - 1, y), v(x, y - 1), h(x, y), v(x, y)]]
    out = ([h(-1, y) for y in range(block)] + [v(x, -1) for x in range(block)]
           + [h(block - 1, y) for y in range(block)] + [v(x, block - 1) for x in range(block)])
    t = np.einsum(*ops, out, optimize="greedy")
    D = 2 ** block
    return np.ascontiguousarray(t.reshape(D, D, D, D))


def uniform_random(chi: int, seed: int, dist: str = "u01+0.1") -> np.ndarray:
    """A uniform tensor of bond dimension chi with entries drawn as
    ``random_tensors`` draws them (one SplitMix64 stream, row-major)."""
    n = chi ** 4
    if dist == "u01+0.1":
        vals = splitmix64_uniform(seed, n) + 0.1
    elif dist == "n1,0.3":
        vals = splitmix64_normal(seed, n, 1.0, 0.3)
    else:
        raise ValueError(dist)
    return vals.reshape(chi, chi, chi, chi).copy()


def uniform_product(a, b, c, e) -> np.ndarray:
    """The rank-1 uniform tensor A[l,u,r,d] = a[l] b[u] c[r] e[d]: every bond
    of its lattice is independent of the others."""
    return np.einsum("i,j,k,l->ijkl", *(np.asarray(x, dtype=np.float64) for x in (a, b, c, e)))


def square_lines(lx: int, ly: int) -> list:
    """Every line between two columns and every line between two rows of an
    lx-by-ly square lattice, as multi-index partitions (the first-level
    partitions of the paper's recursive 4 x 3 example, Sec. IV.A)."""
    return [square_line_x(lx, ly, k) for k in range(lx - 1)] + [square_line_y(lx, ly, k) for k in range(ly - 1)]


def square_block_partitions(lx: int, ly: int, x0: int, y0: int, parts, bw: int = 3, bh: int = 3) -> list:
    """Partitions given on a bw-by-bh square lattice placed at (x0, y0) inside
    an lx-by-ly lattice, with bond ids mapped to the larger lattice."""
    small = square_lattice(bw, bh, 2)
    big = square_lattice(lx, ly, 2)

    def site(s):
        return (y0 + s // bw) * lx + x0 + s % bw
    out = []
    for S in parts:
        out.append(sorted(bond_between(big, site(int(small.bond_site[b][0])), site(int(small.bond_site[b][1])))
                          for b in S))
    return out


def unique_partitions(parts) -> list:
    """The partitions with repeated bond sets dropped (first occurrence kept):
    overlapping blocks can place the same line twice."""
    seen, out = set(), []
    for S in parts:
        key = tuple(sorted(int(b) for b in S))
        if key not in seen:
            seen.add(key)
            out.append(list(key))
    return out

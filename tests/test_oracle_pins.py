"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties an oracle function to something other than itself: a literal
definition (spin sums, subset scans), a textbook closed form (Ising
high-temperature graphs, cycle-space dimension, Onsager), an exact identity of
the paper (Eq. A2-A6 hold for any complementary P, Q) or an invariant.
"""
import math
from collections import Counter

import numpy as np
import pytest

from paper_2512_10910_gb300 import inputs as I
from oracle import bp as B
from oracle import enumerate as E
from oracle import exact as Ex
from oracle import expansion as X


# ---------------------------------------------------------------- exact truth
def test_exact_contractions_agree_with_ising_spin_sum():
    # Eq. A1 three ways vs the definition of Z as a sum over spins.
    g = I.square_lattice(4, 4, 2)
    net = I.ising_tensors(g, 0.40)
    z_spin = Ex.ising_spin_sum(net, 0.40)
    z_ein = float(Ex.contract_einsum(net))
    t, ls = Ex.contract_sweep(net)
    z_sw = float(t) * math.exp(ls)
    assert z_spin == pytest.approx(533158.1721946754, rel=1e-14)
    assert z_ein == pytest.approx(z_spin, rel=1e-13)
    assert z_sw == pytest.approx(z_spin, rel=1e-13)


def test_sweep_matches_einsum_random_and_open():
    g = I.square_lattice(3, 3, 3)
    net = I.random_tensors(g, 3, "bias:0.2")
    t, ls = Ex.contract_sweep(net)
    assert float(t) * math.exp(ls) == pytest.approx(float(Ex.contract_einsum(net)), rel=1e-12)
    go = I.with_open_legs(I.square_lattice(3, 2, 2), [(0, 2), (2, 3), (4, 2)])
    no = I.random_tensors(go, 9)
    t, ls = Ex.contract_sweep(no)
    np.testing.assert_allclose(t * math.exp(ls), Ex.contract_einsum(no), rtol=1e-12)


def test_even_subgraph_counts_cycle_space_and_ht_closed_form():
    # Number of even subgraphs = 2^(M - N + 1) for a connected graph (cycle
    # space dimension), and the high-temperature form reproduces the spin sum.
    for g in (I.square_lattice(4, 4, 2), I.square_lattice(3, 5, 2), I.cubic_lattice(2, 2, 3, 2)):
        cnt = E.even_subsets_by_size(g)
        assert int(cnt.sum()) == 2 ** (g.n_bonds - g.n_sites + 1)
        for beta in (0.2, 0.44, 0.7):
            net = I.ising_tensors(g, beta)
            assert Ex.ising_ht(g.n_sites, g.n_bonds, beta, cnt) == pytest.approx(
                Ex.ising_spin_sum(net, beta), rel=1e-12)
    cnt = E.even_subsets_by_size(I.square_lattice(4, 4, 2))
    assert cnt.tolist()[:21] == [1, 0, 0, 0, 9, 0, 12, 0, 50, 0, 92, 0, 158, 0, 116, 0, 69, 0, 4, 0, 1]


def test_onsager_quadrature_and_exact_corner_estimator():
    # Onsager's closed form vs exact finite lattices (edge/corner terms cancelled).
    b = 0.3
    ons = Ex.onsager_minus_beta_f(b)

    def lnz(lx, ly):
        t, ls = Ex.contract_sweep(I.ising_tensors(I.square_lattice(lx, ly, 2), b))
        return math.log(float(t)) + ls

    errs = [abs(Ex.corner_estimator(lnz(L, L), lnz(L, L - 1), lnz(L - 1, L - 1)) - ons)
            for L in (5, 6, 7)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6
    # infinite-temperature limit: -beta f -> ln 2
    assert Ex.onsager_minus_beta_f(1e-9) == pytest.approx(math.log(2.0), abs=1e-12)


# ---------------------------------------------------------------- enumeration
SMALL_GEOMS = [
    I.square_lattice(3, 3, 2),
    I.square_lattice(2, 4, 2),
    I.cubic_lattice(2, 2, 2, 2),
    # a small irregular graph with a double bond and a triangle
    I.grid_graph(5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 2), (0, 1), (3, 1)], [2] * 8),
]


@pytest.mark.parametrize("gi", range(len(SMALL_GEOMS)))
@pytest.mark.parametrize("mode", [E.LOOP, E.ALL])
@pytest.mark.parametrize("K", [3, 6, 12])
def test_enumerators_agree_with_literal_definition(gi, mode, K):
    g = SMALL_GEOMS[gi]
    lit = E.clusters_python(g, K, mode)
    assert E.clusters_bitmask(g, K, mode) == lit
    assert E.clusters_grow(g, K, mode) == lit


def test_lattice_cluster_counts_closed_forms():
    # On an Lx x Ly square lattice: plaquettes (size 4) = (Lx-1)(Ly-1); size-6
    # loops are 1x2 rectangles; size-7 clusters are the same rectangles with
    # the middle rung (theta graphs): both (Lx-2)(Ly-1) + (Lx-1)(Ly-2).
    for lx, ly in ((5, 4), (7, 6), (16, 16)):
        g = I.square_lattice(lx, ly, 2)
        cnt = Counter(len(c) for c in E.clusters_grow(g, 7, E.LOOP))
        rect = (lx - 2) * (ly - 1) + (lx - 1) * (ly - 2)
        assert cnt[4] == (lx - 1) * (ly - 1)
        assert cnt[6] == rect and cnt[7] == rect
        assert set(cnt) == {4, 6, 7}
    # cubic lattice: plaquettes 3 (L-1)^2 L
    g = I.cubic_lattice(4, 4, 4, 2)
    cnt = Counter(len(c) for c in E.clusters_grow(g, 4, E.LOOP))
    assert cnt == {4: 3 * 3 * 3 * 4}


def test_full_order_loop_counts_4x4():
    # two independent methods on the 4x4 grid at full order
    g = I.square_lattice(4, 4, 2)
    a = E.clusters_bitmask(g, 24, E.LOOP)
    b = E.clusters_grow(g, 12, E.LOOP)
    assert [c for c in a if len(c) <= 12] == b
    assert len(a) == 15593
    assert len(E.enumerate_terms(g, a, 24)) == 16372


def test_terms_are_all_vertex_disjoint_cluster_unions():
    # Every bond set whose components are all LOOP clusters is exactly one term.
    g = I.square_lattice(3, 3, 2)
    K = 12
    cl = E.clusters_python(g, K, E.LOOP)
    idx = {c: i for i, c in enumerate(cl)}
    terms = E.enumerate_terms(g, cl, K)
    from_terms = sorted(tuple(sorted(b for i in t for b in cl[i])) for t in terms)
    lit = []
    for S in E.all_subsets(g, K):
        comps = E.components(g, S)
        if all(c in idx for c in comps):
            lit.append(tuple(sorted(S)))
    assert from_terms == sorted(lit)
    assert len(set(from_terms)) == len(from_terms)


# ---------------------------------------------------------------- BP, projectors
def test_bp_exact_on_a_tree():
    # BP is exact on loop-free networks: Z_BP = prod z_v equals the contraction.
    edges = [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (5, 6)]
    g = I.grid_graph(7, edges, [3, 2, 3, 2, 3, 2])
    net = I.random_tensors(g, 11)
    r = B.bp_fixed_point(net)
    assert r.converged
    proj = B.bond_projectors(net, r)
    z = X.site_values(net, proj)
    assert float(np.prod(z)) == pytest.approx(float(Ex.contract_einsum(net)), rel=1e-12)


def test_ising_bp_fixed_point_is_uniform_and_zbp_closed_form():
    g = I.square_lattice(4, 5, 2)
    beta = 0.35
    net = I.ising_tensors(g, beta)
    r = B.bp_fixed_point(net)
    for m in r.out:
        np.testing.assert_allclose(m, [2 ** -0.5, 2 ** -0.5], atol=1e-15)
    proj = B.bond_projectors(net, r)
    z = X.site_values(net, proj)
    lz = g.n_sites * math.log(2) + g.n_bonds * math.log(math.cosh(beta))
    assert float(np.sum(np.log(z))) == pytest.approx(lz, rel=1e-13)


def test_projectors_are_complementary_rank_one_projectors():
    net = I.random_tensors(I.square_lattice(3, 3, 4), 2)
    r = B.bp_fixed_point(net)
    for P, Q, c0, c1 in B.bond_projectors(net, r):
        np.testing.assert_allclose(P @ P, P, atol=1e-13)
        np.testing.assert_allclose(P + Q, np.eye(4), atol=1e-15)
        assert np.linalg.matrix_rank(P) == 1
        np.testing.assert_allclose(P, np.outer(c0, c1), atol=1e-15)


def test_boundary_reflection_on_open_leg():
    # With the open leg's incoming message equal to its outgoing one, the open
    # message is the normalised dominant solution of a self-consistency; check
    # the fixed-point equation directly on a single site with one open leg.
    go = I.with_open_legs(I.square_lattice(2, 1, 2), [(0, 2)])
    net = I.random_tensors(go, 4)
    r = B.bp_fixed_point(net)
    assert r.converged
    t0 = net.tensors[0]          # legs: bond 0 (to site 1), bond 1 (open)
    k_open = 1
    m_in_bond = r.out[net.site_ptr[1]]      # site 1's message along bond 0
    m_open = r.out[net.site_ptr[0] + k_open]
    upd = np.tensordot(t0, m_in_bond, axes=([0], [0]))
    upd = upd / np.linalg.norm(upd)
    np.testing.assert_allclose(upd * np.sign(upd[np.argmax(np.abs(upd))]), m_open, atol=1e-12)


# ---------------------------------------------------------------- expansion identities
def _random_oblique(net, seed):
    rng = np.random.default_rng(seed)
    proj = []
    for b in range(net.n_bonds):
        d = int(net.bond_dim[b])
        u, v = rng.normal(size=d), rng.normal(size=d)
        v = v / np.dot(u, v)
        P = np.outer(u, v)
        proj.append((P, np.eye(d) - P, u, v))
    return proj


@pytest.mark.parametrize("shape,D", [((2, 2), 3), ((3, 2), 3), ((3, 3), 2)])
def test_full_order_all_mode_is_exact_for_any_projector(shape, D):
    # Eq. A2-A4 and A6 are exact identities for any complementary P, Q.
    net = I.random_tensors(I.square_lattice(shape[0], shape[1], D), 21, "bias:0.2")
    z = float(Ex.contract_einsum(net))
    M = net.n_bonds
    r_bp = X.pne(net, M, E.ALL)
    r_rand = X.pne(net, M, E.ALL, proj=_random_oblique(net, 5))
    assert r_bp.value == pytest.approx(z, rel=1e-11)
    assert r_rand.value == pytest.approx(z, rel=1e-9)
    assert r_bp.n_terms == 2 ** M


def test_linear_and_combinatorial_forms_eq_a4_a6():
    # Literal Eq. A4 (M+1 terms Z(Q^r P I..)) and Eq. A6 (residue plus signed
    # sum over P/I strings) on a 6-bond network with random oblique projectors.
    net = I.random_tensors(I.square_lattice(2, 3, 2), 8, "bias:0.2")
    proj = _random_oblique(net, 1)
    M = net.n_bonds
    z0 = float(Ex.contract_einsum(net))

    def contract(ops_per_bond):
        ops = []
        for v in range(net.n_sites):
            labels = [2 * int(b) + (0 if int(net.bond_site[b][0]) == v else 1) for b in net.legs(v)]
            ops += [net.tensors[v], labels]
        for b in range(M):
            ops += [ops_per_bond[b], [2 * b, 2 * b + 1]]
        return float(np.einsum(*X._compact_labels(ops), [], optimize="greedy"))

    P = [p[0] for p in proj]
    Q = [p[1] for p in proj]
    Id = [np.eye(int(net.bond_dim[b])) for b in range(M)]
    linear = contract(Q) + sum(contract(Q[:r] + [P[r]] + Id[r + 1:]) for r in range(M))
    assert linear == pytest.approx(z0, rel=1e-11)
    comb = contract(Q)
    for x in range(1, 2 ** M):
        ops = [P[b] if (x >> b) & 1 else Id[b] for b in range(M)]
        comb += (1 if bin(x).count("1") % 2 else -1) * contract(ops)
    assert comb == pytest.approx(z0, rel=1e-10)
    # each linear-form term is the sum of the P/Q strings with that prefix
    r = 2
    strings = 0.0
    for x in range(2 ** (M - r - 1)):
        ops = Q[:r] + [P[r]] + [Q[b] if (x >> (b - r - 1)) & 1 else P[b] for b in range(r + 1, M)]
        strings += contract(ops)
    assert strings == pytest.approx(contract(Q[:r] + [P[r]] + Id[r + 1:]), rel=1e-11)


def test_factorised_term_equals_whole_network_contraction():
    net = I.random_tensors(I.square_lattice(3, 2, 3), 5)
    proj = _random_oblique(net, 2)
    z = X.site_values(net, proj)
    for Es in [(0,), (0, 1), (1, 3, 5), (0, 2, 4, 6), tuple(range(7))]:
        comps = E.components(net, Es)
        covered = {v for C in comps for v in E.cluster_vertices(net, C)}
        f = np.prod([z[v] for v in range(net.n_sites) if v not in covered])
        f *= np.prod([X.cluster_value(net, proj, C) for C in comps])
        assert f == pytest.approx(X.term_value_unfactorized(net, proj, Es), rel=1e-12)


def test_dangling_clusters_vanish_at_bp_fixed_point():
    net = I.random_tensors(I.square_lattice(4, 3, 3), 6)
    r = X.pne(net, 4, E.LOOP)  # BP fixed point and its projectors
    proj = r.proj
    z = r.z
    for C in E.clusters_python(net, 3, E.ALL):
        w = X.cluster_value(net, proj, C) / np.prod([z[v] for v in E.cluster_vertices(net, C)])
        assert abs(w) < 1e-11, (C, w)        # every such cluster has a degree-1 site
    # and a loop cluster does not vanish
    plaq = E.clusters_python(net, 4, E.LOOP)[0]
    assert abs(X.cluster_value(net, proj, plaq)) > 1e-6


def test_loop_full_order_equals_exact_at_fixed_point():
    net = I.random_tensors(I.square_lattice(3, 3, 2), 13)
    r = X.pne(net, net.n_bonds, E.LOOP)
    assert r.value == pytest.approx(float(Ex.contract_einsum(net)), rel=1e-11)


def test_ising_loop_expansion_is_the_high_temperature_series():
    # In the paramagnetic BP gauge every cluster weight is tanh(beta)^|C| if
    # all its vertices have even degree, else 0: c_k = n_k tanh^k.
    g = I.square_lattice(3, 4, 2)
    beta = 0.4
    net = I.ising_tensors(g, beta)
    K = g.n_bonds
    r = X.pne(net, K, E.LOOP)
    cnt = E.even_subsets_by_size(g)
    t = math.tanh(beta)
    np.testing.assert_allclose(r.c, [cnt[k] * t ** k for k in range(K + 1)], atol=1e-13)
    assert r.value == pytest.approx(Ex.ising_spin_sum(net, beta), rel=1e-13)
    assert r.log_abs_zref == pytest.approx(g.n_sites * math.log(2) + g.n_bonds * math.log(math.cosh(beta)), rel=1e-14)


def test_pne_log_series_approaches_onsager():
    # The 2D Ising network must approach the Onsager free energy: the
    # corner-cancelled order-K log series converges to it monotonically.
    b = 0.3
    ons = Ex.onsager_minus_beta_f(b)

    def ls(lx, ly, K):
        return X.pne(I.ising_tensors(I.square_lattice(lx, ly, 2), b), K, E.LOOP).log_series

    errs = []
    for K in (4, 6, 8):
        est = Ex.corner_estimator(ls(7, 7, K), ls(7, 6, K), ls(6, 6, K))
        errs.append(ons - est)
    assert errs[0] > errs[1] > errs[2] > 0
    assert errs[2] < 1e-4


def test_scaling_and_gauge_invariance():
    net = I.random_tensors(I.square_lattice(3, 3, 3), 17)
    K = 8
    r0 = X.pne(net, K, E.LOOP)
    # scaling one site tensor by s scales Z_K by s
    t2 = list(net.tensors)
    t2[4] = 2.5 * t2[4]
    r1 = X.pne(net.with_tensors(t2), K, E.LOOP)
    assert r1.log_abs - r0.log_abs == pytest.approx(math.log(2.5), abs=1e-12)
    np.testing.assert_allclose(r1.c, r0.c, atol=1e-13)
    # a random invertible gauge on bond 3 leaves every c_k unchanged
    rng = np.random.default_rng(3)
    G = np.eye(3) + 0.3 * rng.normal(size=(3, 3))
    Gi = np.linalg.inv(G)
    s0, s1 = (int(x) for x in net.bond_site[3])
    t3 = list(net.tensors)
    for v, M in ((s0, G), (s1, Gi.T)):
        ax = list(int(b) for b in net.legs(v)).index(3)
        t3[v] = np.moveaxis(np.tensordot(t3[v], M, axes=([ax], [0])), -1, ax)
    r2 = X.pne(net.with_tensors(t3), K, E.LOOP)
    np.testing.assert_allclose(r2.c, r0.c, atol=1e-11)
    assert r2.log_abs == pytest.approx(r0.log_abs, abs=1e-11)


def test_open_output_full_order_is_exact():
    # Sec. III.D geometry: 2x3 network with three open indices.
    go = I.with_open_legs(I.square_lattice(3, 2, 2), [(0, 2), (2, 2), (4, 2)])
    net = I.random_tensors(go, 12)
    out, _, _ = X.pne_open(net, 99, E.ALL)
    ex = Ex.contract_einsum(net)
    assert Ex.eps2(ex, out) < 1e-12


def test_neumaier_and_power_series_log():
    assert X.neumaier([1e16, 1.0, -1e16]) == 1.0
    assert X.neumaier([0.1] * 10) == 1.0
    a, b = 0.3, -0.7
    c = [1.0, a + b, a * b, 0.0, 0.0, 0.0]       # (1 + a x)(1 + b x)
    l = X.power_series_log(c, 5)
    for k in range(1, 6):
        assert l[k] == pytest.approx((-1) ** (k + 1) * (a ** k + b ** k) / k, rel=1e-14)


def test_golden_count_file_is_the_oracle_output():
    # the stored full-size counts come from the oracle alone: recompute the
    # cheapest entry (the 16x16 bench geometry, K = 8) and compare every field
    import json
    import os
    from collections import Counter
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cluster_counts.json")))
    ref = golden["cases"]["square16x16"]
    g = I.square_lattice(16, 16, 2)
    cl = E.clusters_grow(g, 8, E.LOOP)
    terms = E.enumerate_terms(g, cl, 8)
    assert (len(cl), len(terms)) == (ref["n_clusters"], ref["n_terms"]) == (2827, 27216)
    by_size = Counter(len(c) for c in cl)
    by_order = Counter(sum(len(cl[i]) for i in t) for t in terms)
    assert {str(k): v for k, v in sorted(by_size.items())} == ref["clusters_by_size"]
    assert {str(k): v for k, v in sorted(by_order.items())} == ref["terms_by_order"]

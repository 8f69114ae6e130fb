"""Pins of the combinatorial-form oracle (multi-index partitions, Eq. A6,
Eq. A8-A10), against what the paper and the mathematics fix:

* Eq. A6 (and Eq. A4 over partitions) is an exact identity for ANY
  complementary projectors: the kept sub-networks plus the residue, inserted
  directly as the non-factorising complement of each partition (Eq. A9),
  equal the exact contraction -- random oblique projectors here.
* The 3 x 3 network with six partitions has C(6,2)+...+C(6,6) = 57 sub-leading
  networks (Sec. III.B).
* At a BP fixed point the linear form over the double loop's three vertical
  bonds leaves a single degree-7 loop term as its residue (Sec. III.A): the
  residue inserted directly equals Z_BP w(C) for C = all seven bonds.
* The residue's loop terms by degree, for the 3 x 3 readings of Fig. 4: one
  degree-8 and six degree-10 terms for four single-index partitions; five
  degree-8 terms (and six degree-9) for the six multi-index partitions
  (Sec. III.B).
* At a BP fixed point the combinatorial sum equals the loop series restricted
  to the terms that miss at least one partition (every term meeting all
  partitions is a residue term) -- two independent computations.
"""
import math

import numpy as np
import pytest

from paper_2512_10910_gb300 import inputs as I
from oracle import bp as OB
from oracle import combinatorial as OC
from oracle import enumerate as E
from oracle import exact as Ex
from oracle import expansion as X


def _oblique_projectors(net, seed):
    """Random rank-1 oblique projectors P_b = u v^T / (v . u) on every bond."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(net.n_bonds):
        d = int(net.bond_dim[b])
        u, v = rng.normal(size=d), rng.normal(size=d)
        n = float(v @ u)
        P = np.outer(u, v) / n
        out.append((P, np.eye(d) - P, u, v / n))
    return out


CASES = [
    ("double_loop", lambda: I.random_tensors(I.square_lattice(3, 2, 3), 1, "bias:0.2"), I.double_loop_vertical),
    ("3x3_pinwheel", lambda: I.random_tensors(I.square_lattice(3, 3, 2), 2, "bias:0.2"), I.square3x3_pinwheel),
    ("3x3_six_lines", lambda: I.random_tensors(I.square_lattice(3, 3, 2), 3, "bias:0.2"), I.square3x3_six_lines),
    ("cube2_planes", lambda: I.random_tensors(I.cubic_lattice(2, 2, 2, 2), 4, "bias:0.2"), I.cube2_planes),
]


@pytest.mark.parametrize("name,make,parts", CASES, ids=[c[0] for c in CASES])
def test_eq_a6_and_a4_are_exact_for_any_projectors(name, make, parts):
    net = make()
    partitions = parts()
    proj = _oblique_projectors(net, 11)
    z0 = float(Ex.contract_einsum(net))
    r = OC.combinatorial_pne(net, partitions, proj=proj)
    R = OC.residue_direct(net, partitions, proj)
    assert r["value"] + R == pytest.approx(z0, rel=1e-11, abs=1e-12 * abs(z0))
    assert OC.linear_pne(net, partitions, proj) + R == pytest.approx(z0, rel=1e-11, abs=1e-12 * abs(z0))
    # a dropped sign, a missing sub-network or a wrong complement breaks it
    assert r["n_terms"] == 2 ** len(partitions) - 1


def test_3x3_six_partitions_have_57_subleading_networks():
    subsets = OC.comb_subsets(6)
    assert sum(1 for x, _ in subsets if len(x) >= 2) == 57
    assert sum(1 for x, _ in subsets if len(x) == 1) == 6
    assert all(s == (1 if len(x) % 2 else -1) for x, s in subsets)


def test_partition_complement_does_not_factorise():
    # Eq. A9: Q_ij = Q_i x P_j + P_i x Q_j + Q_i x Q_j, not Q_i x Q_j
    net = I.random_tensors(I.square_lattice(3, 3, 3), 5)
    proj = _oblique_projectors(net, 3)
    S = [0, 1]
    Q = OC.partition_complement(proj, S)
    P0, Q0, P1, Q1 = proj[0][0], proj[0][1], proj[1][0], proj[1][1]
    want = (np.einsum("ac,bd->abcd", Q0, P1) + np.einsum("ac,bd->abcd", P0, Q1) + np.einsum("ac,bd->abcd", Q0, Q1))
    np.testing.assert_allclose(Q, want, atol=1e-12)
    assert np.max(np.abs(Q - np.einsum("ac,bd->abcd", Q0, Q1))) > 1e-3


def _full_order_loop(net):
    """The LOOP-mode loop series of the network to full order (oracle)."""
    return X.pne(net, int(net.n_bonds), E.LOOP)


def test_double_loop_residue_is_the_single_degree_7_term():
    net = I.random_tensors(I.square_lattice(3, 2, 3), 7)
    parts = I.double_loop_vertical()
    ref = _full_order_loop(net)
    proj = ref.proj
    touching = OC.terms_touching_all(ref.clusters, ref.terms, parts)
    by_degree = {}
    for _, deg, all_hit in touching:
        if all_hit:
            by_degree[deg] = by_degree.get(deg, 0) + 1
    assert by_degree == {7: 1}
    # that term is the cluster of all seven bonds; the residue inserted
    # directly (Q on the three vertical bonds) equals Z_BP w(C) for it
    C = tuple(range(net.n_bonds))
    i = list(ref.clusters).index(C)
    zbp = math.exp(ref.log_abs_zref) * ref.sign_zref
    R = OC.residue_direct(net, parts, proj)
    assert R == pytest.approx(zbp * ref.w[i], rel=1e-9, abs=1e-12 * abs(zbp))


def test_3x3_residue_terms_by_degree_match_the_text():
    net = I.random_tensors(I.square_lattice(3, 3, 2), 1)
    ref = _full_order_loop(net)

    def residue_degrees(parts):
        out = {}
        for _, deg, all_hit in OC.terms_touching_all(ref.clusters, ref.terms, parts):
            if all_hit:
                out[deg] = out.get(deg, 0) + 1
        return dict(sorted(out.items()))
    single = residue_degrees(I.square3x3_pinwheel())
    assert min(single) == 8 and single[8] == 1 and single.get(9, 0) == 0 and single[10] == 6
    multi = residue_degrees(I.square3x3_six_lines())
    assert min(multi) == 8 and multi[8] == 5 and multi[9] == 6


# positive tensors (BP converges): entries U[0,1) + 0.1
BP_CASES = [
    ("double_loop", lambda: I.random_tensors(I.square_lattice(3, 2, 3), 1), I.double_loop_vertical),
    ("3x3_six_lines", lambda: I.random_tensors(I.square_lattice(3, 3, 3), 3), I.square3x3_six_lines),
    ("3x3_aklt_six_lines", lambda: I.aklt_tensors(I.square_lattice(3, 3, 4)), I.square3x3_six_lines),
    ("cube2_planes", lambda: I.random_tensors(I.cubic_lattice(2, 2, 2, 2), 4), I.cube2_planes),
]


@pytest.mark.parametrize("name,make,parts", BP_CASES, ids=[c[0] for c in BP_CASES])
def test_combinatorial_sum_is_the_loop_series_without_the_residue_terms(name, make, parts):
    # at a BP fixed point: Z(P^x) = Z_BP * (sum of the loop terms whose excited
    # bonds avoid every partition in x), so the signed sum over x keeps exactly
    # the terms that miss at least one partition
    net = make()
    partitions = parts()
    ref = _full_order_loop(net)
    r = OC.combinatorial_pne(net, partitions, proj=ref.proj)
    zbp = math.exp(ref.log_abs_zref) * ref.sign_zref
    kept = [0.0]
    w = np.asarray(ref.w)
    for t, deg, all_hit in OC.terms_touching_all(ref.clusters, ref.terms, partitions):
        if not all_hit:
            kept.append(float(np.prod([w[i] for i in t])) if t else 1.0)
    loop_value = zbp * X.neumaier(kept)
    assert r["value"] == pytest.approx(loop_value, rel=1e-9)
    # and the full loop series is the exact contraction
    assert ref.value == pytest.approx(float(Ex.contract_einsum(net)), rel=1e-9)

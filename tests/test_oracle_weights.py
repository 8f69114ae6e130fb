"""Pins of the weight-passing oracle and of rank-r expansions (App. C, Sec. V):

* the coarse-grained Ising recipe contracts to the spin sum (4 x 4 lattice in
  2 x 2 blocks) and to the fine lattice's sweep contraction (12 x 12 in 4 x 4
  blocks, bond dimension 16);
* weight passing is a pure change of gauge: the network with the weights
  inserted keeps the exact value; the weights end positive, sorted, largest 1;
* with full-rank projectors (r = d) every term but the first vanishes and the
  expansion is exact; Eq. A4 and A6 stay exact for rank-r projectors;
* the degenerate sub-critical Ising network of Sec. V.B (12 x 12 coarse-grained
  into 3 x 3 with bond dimension 16): rank-1 expansions (BP and weight
  passing) miss by percents below 0.8 T_c, rank-2 weight-passing expansions
  reach a relative error below 1e-7 (both the four single-index partitions
  and the six multi-index partitions of the 3 x 3 network).
"""
import math

import numpy as np
import pytest

from paper_2512_10910_gb300 import inputs as I
from oracle import bp as OB
from oracle import combinatorial as OC
from oracle import exact as Ex
from oracle import weights as OW

BETA_C = math.log(1 + math.sqrt(2)) / 2


def test_blocked_ising_recipe_contracts_to_the_spin_sum():
    net = I.ising_blocked(2, 2, 2, 0.4)
    assert list(net.bond_dim) == [4, 4, 4, 4]
    z = Ex.ising_spin_sum(I.ising_tensors(I.square_lattice(4, 4, 2), 0.4), 0.4)
    assert float(Ex.contract_einsum(net)) == pytest.approx(z, rel=1e-13)
    big = I.ising_blocked(3, 3, 4, 0.5)
    t, ls = Ex.contract_sweep(I.ising_tensors(I.square_lattice(12, 12, 2), 0.5))
    assert math.log(float(Ex.contract_einsum(big))) == pytest.approx(math.log(float(t)) + ls, abs=1e-12)


@pytest.mark.parametrize("make", [lambda: I.random_tensors(I.square_lattice(3, 3, 3), 4),
                                  lambda: I.ising_blocked(3, 3, 2, 0.55),
                                  lambda: I.random_tensors(I.cubic_lattice(2, 2, 2, 3), 6)])
def test_weight_passing_is_a_change_of_gauge(make):
    net = make()
    z0 = float(Ex.contract_einsum(net))
    tens, S, ls, sweeps, change = OW.weight_passing(net, 0.8, 1e-11, 3000)
    assert change < 1e-11
    for s in S:
        assert np.all(s > 0) and s[0] == 1.0 and np.all(np.diff(s) <= 1e-15)
    wn, ls = OW.weighted_network(net, tens, S, ls)
    assert float(Ex.contract_einsum(wn)) * math.exp(ls) == pytest.approx(z0, rel=1e-8)


def test_full_rank_projectors_make_the_expansion_exact_and_identities_hold():
    net = I.random_tensors(I.square_lattice(3, 3, 3), 8)
    z0 = float(Ex.contract_einsum(net))
    tens, S, ls, _, _ = OW.weight_passing(net, 0.8, 1e-11, 3000)
    wn, ls = OW.weighted_network(net, tens, S, ls)
    full = OW.rank_r_projectors(wn, 3)
    assert OW.rank_r_linear(wn, I.square3x3_pinwheel(), full) * math.exp(ls) == pytest.approx(z0, rel=1e-9)
    # Eq. A4 / A6 with rank-r projectors and the complements inserted directly
    # (bond dimension 3, rank 2: the complement has rank 1)
    for r in (1, 2):
        proj = OW.rank_r_projectors(wn, r)
        parts = I.square3x3_pinwheel()
        R = OC.residue_direct(wn, parts, proj)
        zw = z0 / math.exp(ls)
        assert OW.rank_r_linear(wn, parts, proj) + R == pytest.approx(zw, rel=1e-9)
        assert OW.rank_r_combinatorial(wn, parts, proj) + R == pytest.approx(zw, rel=1e-9)
    # multi-index partitions (joint complements of up to four bonds) at D = 2
    net = I.random_tensors(I.square_lattice(3, 3, 2), 9)
    z0 = float(Ex.contract_einsum(net))
    tens, S, ls, _, _ = OW.weight_passing(net, 0.8, 1e-11, 3000)
    wn, ls = OW.weighted_network(net, tens, S, ls)
    for r in (1,):
        proj = OW.rank_r_projectors(wn, r)
        for parts in (I.square3x3_pinwheel(), I.square3x3_six_lines()):
            R = OC.residue_direct(wn, parts, proj)
            lin = OW.rank_r_linear(wn, parts, proj)
            comb = OW.rank_r_combinatorial(wn, parts, proj)
            zw = z0 / math.exp(ls)
            assert lin + R == pytest.approx(zw, rel=1e-9)
            assert comb + R == pytest.approx(zw, rel=1e-9)


@pytest.mark.parametrize("frac", [0.6, 0.7])
def test_degenerate_ising_needs_rank_two(frac):
    beta = BETA_C / frac                               # T = frac * T_c, below 0.8 T_c
    net = I.ising_blocked(3, 3, 4, beta)
    z0 = float(Ex.contract_einsum(net))
    tens, S, ls, _, change = OW.weight_passing(net, 0.8, 1e-10, 3000)
    assert change < 1e-10
    wn, ls = OW.weighted_network(net, tens, S, ls)
    single, multi = I.square3x3_pinwheel(), I.square3x3_six_lines()
    err = {}
    for r in (1, 2):
        proj = OW.rank_r_projectors(wn, r)
        err[("lin", r)] = abs(OW.rank_r_linear(wn, single, proj) * math.exp(ls) / z0 - 1)
        err[("comb", r)] = abs(OW.rank_r_combinatorial(wn, multi, proj) * math.exp(ls) / z0 - 1)
    bp = OB.bp_fixed_point(net, max_iter=20000)
    assert bp.converged
    bp_comb = abs(OC.combinatorial_pne(net, multi, proj=OB.bond_projectors(net, bp))["value"] / z0 - 1)
    assert err[("lin", 1)] > 1e-2 and err[("comb", 1)] > 1e-1 and bp_comb > 1e-1
    assert err[("lin", 2)] < 1e-7 and err[("comb", 2)] < 1e-7

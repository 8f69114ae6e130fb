"""Pins of the recursive-partitioning oracle (Sec. IV.A): with every
second-level residue added back it equals the one-level combinatorial form
exactly (Eq. A6 holds at each level); with a threshold no sub-network exceeds
it is the one-level form; the sub-networks it expands again are the ones the
geometry says (the paper's 4 x 3 example: every line between columns and
rows, the 3 x 3 expansion of Fig. 4 on each 3 x 3 block)."""
import numpy as np

from paper_2512_10910_gb300 import inputs as I
from oracle import exact as X
from oracle import recursive as R
from oracle import weights as OW


def _setup(d, seed=5):
    net = I.random_tensors(I.square_lattice(4, 3, d), seed)
    tens, S, ls, sw, ch = OW.weight_passing(net, 0.8, 1e-11, 5000)
    wn, _ = OW.weighted_network(net, tens, S, ls)
    proj = OW.rank_r_projectors(wn, 1)
    p1 = I.square_lines(4, 3)
    p2 = I.unique_partitions(I.square_block_partitions(4, 3, 0, 0, I.square3x3_six_lines())
                             + I.square_block_partitions(4, 3, 1, 0, I.square3x3_six_lines()))
    return wn, proj, p1, p2


def test_components_of_a_cut_grid():
    g = I.square_lattice(4, 3, 2)
    comps = R.components(g, set(I.square_line_x(4, 3, 0)))
    assert comps == [[0, 4, 8], [1, 2, 3, 5, 6, 7, 9, 10, 11]]
    comps = R.components(g, set(I.square_line_x(4, 3, 1)) | set(I.square_line_y(4, 3, 0)))
    assert sorted(len(c) for c in comps) == [2, 2, 4, 4]


def test_second_level_residues_restore_the_one_level_form():
    wn, proj, p1, p2 = _setup(2)
    plain = OW.rank_r_combinatorial(wn, p1, proj)
    rr = R.recursive_combinatorial(wn, p1, p2, proj, 4, 2, with_residue2=True)
    assert abs(rr["value"] - plain) <= 1e-12 * abs(plain)


def test_threshold_above_every_component_is_the_one_level_form():
    wn, proj, p1, p2 = _setup(3)
    plain = OW.rank_r_combinatorial(wn, p1, proj)
    r = R.recursive_combinatorial(wn, p1, p2, proj, 4, 3)
    assert r["expanded"] == [] and r["contractions"] == 31
    assert abs(r["value"] - plain) <= 1e-13 * abs(plain)


def test_expanded_sub_networks_follow_the_geometry():
    # strips at most 2 wide are cheap: a single outer column line leaves a
    # 3 x 3 block (both sides 3: expanded again), a row line leaves 4 x 1 and
    # 4 x 2 strips, the middle column line two 2 x 3 strips; no sub-network of
    # two or more lines keeps a 3 x 3 block.  Inside columns 1-3 the six lines
    # of that block fit (63 sub-networks); inside columns 0-2 the six lines of
    # its block and the corner line of the other block around site 1 (127)
    wn, proj, p1, p2 = _setup(3)
    r = R.recursive_combinatorial(wn, p1, p2, proj, 4, 2)
    assert r["expanded"] == [(0,), (2,)]
    assert r["contractions"] == 29 + 63 + 127
    exact = float(X.contract_einsum(wn))
    assert abs(r["value"] / exact - 1) < 0.05

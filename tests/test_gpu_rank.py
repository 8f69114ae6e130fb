"""Weight passing (App. C) and rank-r expansions (Sec. V) on the GPU against
the FP64 oracle.

Tolerances: the weights of every bond within 1e-9 of the oracle's (both follow
the same sweep order and update formulas); expansion values within 1e-9
relative of the oracle's own expansion on its own weights (the two gauges
differ only by the signs of singular vectors, which the projectors onto the
largest weights do not see); and, on the degenerate sub-critical Ising network
of Sec. V.B, the rank-2 expansions within 1e-7 of the exact value.
"""
import math

import numpy as np
import pytest

from paper_2512_10910_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2512_10910_gb300 import pne  # noqa: E402
from oracle import exact as Ex  # noqa: E402
from oracle import weights as OW  # noqa: E402

BETA_C = math.log(1 + math.sqrt(2)) / 2


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2512_10910_gb300 import build
    build.build()
    c = pne.Context(0)
    yield c
    c.close()


CASES = [
    ("random3x3_D3", lambda: I.random_tensors(I.square_lattice(3, 3, 3), 4), 2),
    ("random3x3_D4", lambda: I.random_tensors(I.square_lattice(3, 3, 4), 11), 2),
    ("ising3x3_blocked4_0.9Tc", lambda: I.ising_blocked(3, 3, 4, BETA_C / 0.9), 2),
    ("random2x2x2_D3", lambda: I.random_tensors(I.cubic_lattice(2, 2, 2, 3), 6), 1),
]


@pytest.mark.parametrize("name,make,rank", CASES, ids=[c[0] for c in CASES])
def test_weights_and_rank_r_expansions_match_oracle(ctx, name, make, rank):
    net = make()
    tens, S, ls, sweeps, change = OW.weight_passing(net, 0.8, 1e-11, 5000)
    wn, ls = OW.weighted_network(net, tens, S, ls)
    if net.n_sites == 9:
        parts_lin, parts_comb = I.square3x3_pinwheel(), I.square3x3_six_lines()
    else:
        parts_lin, parts_comb = [[0], [5], [9]], I.cube2_planes()
    for form, parts in ((0, parts_lin), (1, parts_comb)):
        (res,), wts, sw, gls = ctx.rank_r(net, parts, rank, form, alpha=0.8, tol=1e-11)
        assert sw[0] == sweeps
        for b in range(net.n_bonds):
            d = int(net.bond_dim[b])
            np.testing.assert_allclose(wts[0, b, :d], S[b], rtol=0, atol=1e-9)
        proj = OW.rank_r_projectors(wn, rank)
        ref = (OW.rank_r_linear if form == 0 else OW.rank_r_combinatorial)(wn, parts, proj)
        lz = math.log(abs(ref)) + ls
        assert abs(res["log_abs"] - lz) <= 1e-9, (form, res["log_abs"], lz)
        assert res["sign"] == (1 if ref > 0 else -1)


@pytest.mark.parametrize("frac", [0.6, 0.7])
def test_degenerate_ising_rank_two_on_gpu(ctx, frac):
    net = I.ising_blocked(3, 3, 4, BETA_C / frac)
    z0 = math.log(float(Ex.contract_einsum(net)))
    for form, parts in ((0, I.square3x3_pinwheel()), (1, I.square3x3_six_lines())):
        (r2,), _, sw, _ = ctx.rank_r(net, parts, 2, form, alpha=0.8, tol=1e-10)
        assert sw[0] > 0
        assert abs(math.expm1(r2["log_abs"] - z0)) < 1e-7
        (r1,), _, _, _ = ctx.rank_r(net, parts, 1, form, alpha=0.8, tol=1e-10)
        assert abs(math.expm1(r1["log_abs"] - z0)) > 1e-2


def test_rank_r_batch_of_tensor_sets(ctx):
    g = I.square_lattice(3, 3, 3)
    nets = [I.random_tensors(g, s) for s in (31, 32, 33)]
    data = np.concatenate([n.flat_data()[0] for n in nets])
    res, wts, sw, ls = ctx.rank_r(nets[0], I.square3x3_pinwheel(), 2, 0, data=data, n_batch=3, tol=1e-11)
    for b, n in enumerate(nets):
        (one,), _, _, _ = ctx.rank_r(n, I.square3x3_pinwheel(), 2, 0, tol=1e-11)
        assert one["log_abs"] == pytest.approx(res[b]["log_abs"], abs=1e-12)


@pytest.mark.parametrize("name,make,rank", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_rank_r_terms_as_grid_gemms(ctx, name, make, rank):
    # the same expansion with every term contracted row by row as GEMMs: FP64
    # equals the site-by-site FP64 path within 1e-10; TF32 / BF16 on the tensor
    # cores within the stated bound of it
    net = make()
    for form, parts in ((0, I.square3x3_pinwheel()), (1, I.square3x3_six_lines())):
        (ref,), _, _, _ = ctx.rank_r(net, parts, rank, form, alpha=0.8, tol=1e-11)
        (g64,), _, _, _ = ctx.rank_r(net, parts, rank, form, alpha=0.8, tol=1e-11, grid=(3, 3), dtype=pne.PNE_F64)
        assert abs(g64["log_abs"] - ref["log_abs"]) <= 1e-10 and g64["sign"] == ref["sign"]
        assert g64["n_terms"] == ref["n_terms"]
        np.testing.assert_allclose(g64["c"], ref["c"], rtol=1e-9, atol=1e-12 * float(np.max(ref["abs_c"])))
        # the weighted network carries signs (gauge transforms), so a term's
        # absolute contraction can exceed |value| and the stated bound is
        # first-order per |value|: checked beside a fixed tolerance per dtype
        for dt, tol in ((pne.PNE_TF32, 1e-2), (pne.PNE_BF16, 5e-2)):
            (r,), _, _, _ = ctx.rank_r(net, parts, rank, form, alpha=0.8, tol=1e-11, grid=(3, 3), dtype=dt)
            err = abs(math.expm1(r["log_abs"] - ref["log_abs"]))
            assert math.isfinite(r["err_bound"]) and r["err_bound"] > 0
            assert err <= max(tol, r["err_bound"]), (name, form, dt, err, r["err_bound"])
            assert err <= tol, (name, form, dt, err)


def test_degenerate_ising_rank_two_grid_fp64_reaches_the_target(ctx):
    net = I.ising_blocked(3, 3, 4, BETA_C / 0.6)
    z0 = math.log(float(Ex.contract_einsum(net)))
    for form, parts in ((0, I.square3x3_pinwheel()), (1, I.square3x3_six_lines())):
        (r2,), _, _, _ = ctx.rank_r(net, parts, 2, form, alpha=0.8, tol=1e-10, grid=(3, 3), dtype=pne.PNE_F64)
        assert abs(math.expm1(r2["log_abs"] - z0)) < 1e-7


def test_recursive_partitioning_matches_oracle(ctx):
    # the paper's 4 x 3 example: every column and row line first, the 3 x 3
    # expansion of Fig. 4 on each 3 x 3 block second, strips at most 2 wide
    # contracted as they are; rank-1 projectors of the weights
    from oracle import recursive as OR
    net = I.random_tensors(I.square_lattice(4, 3, 3), 5)
    p1 = I.square_lines(4, 3)
    p2 = I.unique_partitions(I.square_block_partitions(4, 3, 0, 0, I.square3x3_six_lines())
                             + I.square_block_partitions(4, 3, 1, 0, I.square3x3_six_lines()))
    tens, S, ls, sweeps, change = OW.weight_passing(net, 0.8, 1e-11, 5000)
    wn, ls = OW.weighted_network(net, tens, S, ls)
    proj = OW.rank_r_projectors(wn, 1)
    ns, keep = pne.network_struct(net)
    w = pne.pne_weight_passing(ctx.h, ns, 0.8, 1e-11, 5000)
    try:
        for max_side, dt in ((2, pne.PNE_F64), (3, pne.PNE_F64), (1, pne.PNE_F64), (2, pne.PNE_TF32)):
            ref = OR.recursive_combinatorial(wn, p1, p2, proj, 4, max_side)
            (res,), n = pne.pne_recursive_expand_grid(ctx.h, w, 1, p1, p2, max_side, 1, 4, 3, dt)
            assert n == ref["contractions"]
            lz = math.log(abs(ref["value"])) + ls
            tol = 1e-9 if dt == pne.PNE_F64 else 1e-2
            assert abs(res["log_abs"] - lz) <= tol, (max_side, dt, res["log_abs"], lz)
            assert res["sign"] == (1 if ref["value"] > 0 else -1)
    finally:
        pne.pne_weights_destroy(w)
        del keep

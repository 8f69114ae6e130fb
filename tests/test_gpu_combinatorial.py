"""Combinatorial form over multi-index partitions (Eq. A6, A8-A10) on the GPU
against the FP64 oracle, which contracts every sub-network as written.

Tolerances: term counts exact (2^M - 1 sub-networks); FP64 values within
1e-10 relative on the signed sum and per order within 1e-10 of sum_k |c_k|
(both sides converge BP to 1e-13); FP32 / TF32 / BF16 within the library's
stated a-priori bound.
"""
import math

import numpy as np
import pytest

from paper_2512_10910_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2512_10910_gb300 import pne  # noqa: E402
from oracle import combinatorial as OC  # noqa: E402
from oracle import exact as Ex  # noqa: E402


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
    ("double_loop_D3", lambda: I.random_tensors(I.square_lattice(3, 2, 3), 1), I.double_loop_vertical),
    ("3x3_pinwheel_D3", lambda: I.random_tensors(I.square_lattice(3, 3, 3), 2), I.square3x3_pinwheel),
    ("3x3_six_lines_D4", lambda: I.random_tensors(I.square_lattice(3, 3, 4), 3), I.square3x3_six_lines),
    ("3x3_aklt_six_lines", lambda: I.aklt_tensors(I.square_lattice(3, 3, 4)), I.square3x3_six_lines),
    ("3x3_ising_six_lines", lambda: I.ising_tensors(I.square_lattice(3, 3, 2), 0.4407), I.square3x3_six_lines),
    ("cube2_planes_D3", lambda: I.random_tensors(I.cubic_lattice(2, 2, 2, 3), 4), I.cube2_planes),
    ("4x4_lines_D3", lambda: I.random_tensors(I.square_lattice(4, 4, 3), 5),
     lambda: [I.square_line_x(4, 4, k) for k in range(3)] + [I.square_line_y(4, 4, k) for k in range(3)]),
]


def _check(res, ref, M, tol=1e-10):
    assert res["n_terms"] == 2 ** M - 1
    rel = abs(math.expm1(res["log_abs"] - math.log(abs(ref["value"]))))
    assert res["sign"] == (1 if ref["value"] > 0 else -1)
    assert rel <= tol, rel
    scale = float(np.sum(np.abs(ref["c"])))
    np.testing.assert_allclose(res["c"][:M + 1], ref["c"], rtol=0, atol=tol * scale)


@pytest.mark.parametrize("name,make,parts", CASES, ids=[c[0] for c in CASES])
def test_combinatorial_f64_matches_oracle(ctx, name, make, parts):
    net = make()
    partitions = parts()
    ref = OC.combinatorial_pne(net, partitions)
    (res,) = ctx.combinatorial(net, partitions, pne.PNE_F64)
    _check(res, ref, len(partitions))
    # the neglected residue is all that separates it from the exact value
    R = OC.residue_direct(net, partitions, ref["proj"]) if max(len(S) for S in partitions) <= 1 else None
    if R is not None:
        assert res["value"] + R == pytest.approx(float(Ex.contract_einsum(net)), rel=1e-9)


def test_combinatorial_float_float_bp_and_tensor_sets(ctx):
    # two tensor sets of one geometry, BP in float-float arithmetic
    g = I.square_lattice(3, 3, 3)
    nets = [I.random_tensors(g, s) for s in (21, 22)]
    parts = I.square3x3_six_lines()
    data = np.concatenate([n.flat_data()[0] for n in nets])
    res = ctx.combinatorial(nets[0], parts, pne.PNE_F64, data=data, n_batch=2, arithmetic=1)
    for r, n in zip(res, nets):
        _check(r, OC.combinatorial_pne(n, parts), len(parts))


@pytest.mark.parametrize("dtype", ["f32", "tf32", "bf16"])
def test_combinatorial_reduced_precision_within_stated_bound(ctx, dtype):
    net = I.random_tensors(I.square_lattice(3, 3, 4), 3)
    parts = I.square3x3_six_lines()
    ref = OC.combinatorial_pne(net, parts)
    (res,) = ctx.combinatorial(net, parts, dtype)
    rel = abs(math.expm1(res["log_abs"] - math.log(abs(ref["value"]))))
    assert rel <= res["err_bound"], (rel, res["err_bound"])
    # the 63 sub-networks are each of the size of Z and enter with alternating
    # signs, so the stated bound carries the cancellation factor sum|c|/|sum|:
    # FP32 keeps it small, TF32 and BF16 do not (the bound says so)
    if dtype == "f32":
        assert res["err_bound"] < 1e-4
    else:
        assert res["err_bound"] > 1e-2


def test_combinatorial_components_are_the_kept_bond_components(ctx):
    # the components the library lists: for every sub-network, the connected
    # components of the bonds left after cutting its partitions; checked on
    # the host from the partition sets
    net = I.random_tensors(I.square_lattice(3, 3, 2), 9)
    parts = I.square3x3_six_lines()
    (res,), (edges, w) = ctx.combinatorial(net, parts, pne.PNE_F64, export=True)
    got = {tuple(int(b) for b in row if b >= 0) for row in edges}
    want = set()
    for x, _ in OC.comb_subsets(len(parts)):
        cut = {b for p in x for b in parts[p]}
        kept = [b for b in range(net.n_bonds) if b not in cut]
        # union-find over sites
        par = list(range(net.n_sites))

        def f(a):
            while par[a] != a:
                a = par[a]
            return a
        for b in kept:
            u, v = (int(s) for s in net.bond_site[b])
            par[f(u)] = f(v)
        groups = {}
        for b in kept:
            groups.setdefault(f(int(net.bond_site[b][0])), []).append(b)
        want |= {tuple(sorted(g)) for g in groups.values()}
    assert got == want
    assert res["n_clusters"] == len(want)


def test_combinatorial_rejects_bad_partitions(ctx):
    net = I.random_tensors(I.square_lattice(3, 3, 2), 9)
    for parts in ([[]], [[99]], [[0]] * 21):
        with pytest.raises(pne.PneError) as e:
            ctx.combinatorial(net, parts, pne.PNE_F64)
        assert e.value.status == pne.PNE_EINVAL

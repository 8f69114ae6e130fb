"""GPU path (C ABI) vs the FP64 CPU oracle, element by element.

Tolerances: counts and cluster lists bit-exact; FP64 values within 1e-10
relative on Z_K (|d ln Z| <= 1e-10) and per order within 1e-10 of sum_k |c_k|;
FP64 cluster weights within rtol 1e-10 (atol 1e-13; both sides converge BP to
1e-13).  Reduced precisions: every cluster weight within gamma(n_C) u of its
size class's scale, and Z_K within the library's a-priori bound err_bound.
"""
import math

import numpy as np
import pytest

from paper_2512_10910_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2512_10910_gb300 import pne  # noqa: E402
from oracle import enumerate as E  # noqa: E402
from oracle import exact as Ex  # noqa: E402
from oracle import expansion as X  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2512_10910_gb300 import build
    build.build()
    c = pne.Context(0)
    yield c
    c.close()


def _canon(edges, w):
    tuples = [tuple(int(x) for x in r if x >= 0) for r in edges]
    order = sorted(range(len(tuples)), key=lambda i: (len(tuples[i]), tuples[i]))
    return [tuples[i] for i in order], (w[:, order] if w is not None else None)


def _check_values(res, ref, tol=1e-10):
    assert abs(res["log_abs"] - ref.log_abs) <= tol, (res["log_abs"], ref.log_abs)
    assert res["sign"] == ref.sign
    scale = float(np.sum(np.abs(ref.c)))
    np.testing.assert_allclose(res["c"], ref.c, rtol=0, atol=tol * scale)


# ---------------------------------------------------------------- closed-form pins
def test_ising_4x4_full_order_loop_equals_brute_force(ctx):
    net = I.ising_tensors(I.square_lattice(4, 4, 2), 0.40)
    (res,), (edges, w) = ctx.expand(net, 24, pne.PNE_MODE_LOOP, pne.PNE_F64, export=True)
    z = Ex.ising_spin_sum(net, 0.40)
    assert res["value"] == pytest.approx(z, rel=1e-12)
    assert res["n_clusters"] == 15593 and res["n_terms"] == 16372
    cl, _ = _canon(edges, None)
    assert cl == E.clusters_bitmask(net, 24, E.LOOP)
    cnt = E.even_subsets_by_size(net)
    t = math.tanh(0.40)
    np.testing.assert_allclose(res["c"], [cnt[k] * t ** k for k in range(25)], atol=1e-13)


def test_ising_4x4_full_order_all_mode(ctx):
    net = I.ising_tensors(I.square_lattice(4, 4, 2), 0.40)
    (res,) = ctx.expand(net, 24, pne.PNE_MODE_ALL, pne.PNE_F64)
    assert res["value"] == pytest.approx(Ex.ising_spin_sum(net, 0.40), rel=1e-12)
    assert res["n_terms"] == 2 ** 24
    assert res["n_clusters"] == E.count_clusters_bitmask(net, 24, E.ALL)


def test_all_mode_random_full_order_is_exact(ctx):
    # Eq. A2-A4: summing every P/Q string reproduces the network, whatever P is.
    net = I.random_tensors(I.square_lattice(3, 3, 2), 4, "bias:0.2")
    (res,) = ctx.expand(net, 12, pne.PNE_MODE_ALL, pne.PNE_F64)
    assert res["value"] == pytest.approx(float(Ex.contract_einsum(net)), rel=1e-11)
    ref = X.pne(net, 12, E.ALL)
    _check_values(res, ref)


@pytest.mark.parametrize("shape,D,seed", [((3, 3), 3, 1), ((2, 3), 3, 2), ((3, 3), 2, 3), ((2, 4), 4, 5)])
def test_loop_full_order_is_exact_at_fixed_point(ctx, shape, D, seed):
    net = I.random_tensors(I.square_lattice(shape[0], shape[1], D), seed)
    M = net.n_bonds
    (res,) = ctx.expand(net, M, pne.PNE_MODE_LOOP, pne.PNE_F64)
    assert res["value"] == pytest.approx(float(Ex.contract_einsum(net)), rel=1e-10)
    _check_values(res, X.pne(net, M, E.LOOP))


# ---------------------------------------------------------------- oracle parity
@pytest.mark.parametrize("L,D,K,seed", [(6, 4, 8, 0), (5, 3, 10, 7), (7, 5, 6, 3), (16, 4, 8, 0)])
def test_random_2d_parity_f64(ctx, L, D, K, seed):
    net = I.random_tensors(I.square_lattice(L, L, D), seed)
    ref = X.pne(net, K, E.LOOP)
    (res,), (edges, w) = ctx.expand(net, K, pne.PNE_MODE_LOOP, pne.PNE_F64, export=True)
    assert res["n_clusters"] == ref.n_clusters and res["n_terms"] == ref.n_terms
    cl, wc = _canon(edges, w)
    assert cl == list(ref.clusters)
    np.testing.assert_allclose(wc[0], ref.w, rtol=1e-10, atol=1e-13)
    _check_values(res, ref)


def test_cubic_parity_and_batch(ctx):
    g = I.cubic_lattice(3, 3, 3, 2)
    nets = [I.ising_tensors(g, b) for b in (0.20, 0.2217, 0.25)] + [I.random_tensors(g, 9, "n1,0.3")]
    data = np.concatenate([n.flat_data()[0] for n in nets])
    res = ctx.expand(nets[0], 8, pne.PNE_MODE_LOOP, pne.PNE_F64, data=data, n_batch=len(nets))
    for r, n in zip(res, nets):
        ref = X.pne(n, 8, E.LOOP)
        assert r["n_clusters"] == ref.n_clusters and r["n_terms"] == ref.n_terms
        _check_values(r, ref)


def test_batch_equals_individual_bitwise(ctx):
    g = I.square_lattice(6, 5, 4)
    nets = [I.random_tensors(g, s) for s in (11, 12, 13)]
    data = np.concatenate([n.flat_data()[0] for n in nets])
    batch = ctx.expand(nets[0], 8, pne.PNE_MODE_LOOP, pne.PNE_F64, data=data, n_batch=3)
    for r, n in zip(batch, nets):
        (one,) = ctx.expand(n, 8, pne.PNE_MODE_LOOP, pne.PNE_F64)
        assert np.array_equal(one["c"], r["c"]) and one["log_abs"] == r["log_abs"]


def test_deterministic_and_device_input(ctx):
    net = I.random_tensors(I.square_lattice(8, 8, 4), 21)
    flat, _ = net.flat_data()
    (a,) = ctx.expand(net, 8, pne.PNE_MODE_LOOP, pne.PNE_F64)
    (b,) = ctx.expand(net, 8, pne.PNE_MODE_LOOP, pne.PNE_F64, data=torch.from_numpy(flat).cuda())
    assert np.array_equal(a["c"], b["c"]) and a["log_abs"] == b["log_abs"]


# unit roundoff of the contraction dtype (TF32 and BF16: operands rounded,
# FP32 accumulation)
UNIT = {"f32": 2.0 ** -24, "tf32": 2.0 ** -11, "bf16": 2.0 ** -8}
# the stated a-priori bound on Z_K must itself be small (not vacuous)
BOUND_CAP = {"f32": 1e-5, "tf32": 2e-2, "bf16": 1e-1}


def _check_dtype_elementwise(ctx, net, K, dtype):
    """Reduced-precision cluster values against the FP64 oracle, cluster by
    cluster, and Z_K against the library's stated bound.

    A cluster contraction rounds every site factor it reads and every entry
    of its running tensor once in the working dtype, n_C = 2 (|V(C)| + |C|)
    roundings along any product path, so its forward error is at most
    gamma(n_C) u times the contraction of absolute values.  That absolute
    contraction is bounded here by the largest |w| among the clusters of the
    same size (a normwise bound per size class; values that cancel to near
    zero are held to the class's scale, not to their own; a class that
    vanishes altogether is held to the largest weight of any class).
    """
    u = UNIT[dtype]
    ref = X.pne(net, K, E.LOOP)
    (res,), (edges, w) = ctx.expand(net, K, pne.PNE_MODE_LOOP, dtype, export=True)
    assert res["n_clusters"] == ref.n_clusters and res["n_terms"] == ref.n_terms
    cl, wc = _canon(edges, w)
    assert cl == list(ref.clusters)
    wo, wg = np.asarray(ref.w), wc[0]
    sizes = np.array([len(c) for c in cl])
    nverts = np.array([len({int(v) for b in c for v in net.bond_site[b]}) for c in cl])
    n = 2 * (nverts + sizes)
    gam = n * u / (1 - n * u)
    top = float(np.max(np.abs(wo)))
    for k in np.unique(sizes):
        m = sizes == k
        scale = float(np.max(np.abs(wo[m])))
        if scale <= 1e-12 * top:
            # a class that vanishes (odd-degree clusters of the Ising and AKLT
            # networks, zero by symmetry up to FP64 rounding) is held to the
            # largest weight of any class
            scale = top
        err = np.abs(wg[m] - wo[m])
        assert np.all(err <= gam[m] * scale), (dtype, int(k), float(np.max(err / (gam[m] * scale))))
    rel = abs(math.expm1(res["log_abs"] - ref.log_abs))
    assert res["err_bound"] <= BOUND_CAP[dtype], res["err_bound"]
    assert rel <= res["err_bound"], (rel, res["err_bound"])
    return rel, res["err_bound"]


@pytest.mark.parametrize("dtype", ["f32", "tf32", "bf16"])
@pytest.mark.parametrize("case", ["random2d", "aklt", "random3d"])
def test_reduced_precision_cluster_values_and_bound(ctx, dtype, case):
    if case == "random2d":
        net, K = I.random_tensors(I.square_lattice(8, 8, 4), 3), 8
    elif case == "aklt":
        net, K = I.aklt_tensors(I.square_lattice(6, 6, 4)), 8
    else:
        net, K = I.random_tensors(I.cubic_lattice(4, 4, 4, 3), 2, "n1,0.3"), 6
    rel, bound = _check_dtype_elementwise(ctx, net, K, dtype)
    print(case, dtype, "rel err", rel, "bound", bound)


@pytest.mark.parametrize("dtype", ["f32", "tf32", "bf16"])
def test_reduced_precision_ising_cubic(ctx, dtype):
    # q = 1: one number per site, a cluster is a plain product (no cancellation)
    net = I.ising_tensors(I.cubic_lattice(4, 4, 4, 2), 0.2217)
    _check_dtype_elementwise(ctx, net, 8, dtype)


# ---------------------------------------------------------------- open indices
def test_open_output_all_mode_exact(ctx):
    go = I.with_open_legs(I.square_lattice(3, 2, 2), [(0, 2), (2, 2), (4, 2)])
    net = I.random_tensors(go, 12)
    mant, ls = ctx.open_tensor(net, 7, pne.PNE_MODE_ALL, pne.PNE_F64)   # 7 closed bonds: full order
    T = mant[0] * math.exp(ls[0])                                       # through pne_open_tensor
    assert np.max(np.abs(mant)) == pytest.approx(1.0)
    assert Ex.eps2(Ex.contract_einsum(net), T) < 1e-12


def test_open_output_loop_parity(ctx):
    go = I.with_open_legs(I.square_lattice(4, 3, 3), [(0, 2), (5, 3), (11, 2)])
    net = I.random_tensors(go, 5)
    ref, entries, _ = X.pne_open(net, 8, E.LOOP)
    mant, ls = ctx.open_tensor(net, 8, pne.PNE_MODE_LOOP, pne.PNE_F64)
    T = mant[0] * math.exp(ls[0])                                       # through pne_open_tensor
    np.testing.assert_allclose(T, ref, rtol=1e-10)
    # two tensor sets at once: set-major output, one scale per set
    net2 = I.random_tensors(go, 6)
    data = np.concatenate([net.flat_data()[0], net2.flat_data()[0]])
    mant2, ls2 = ctx.open_tensor(net, 8, pne.PNE_MODE_LOOP, pne.PNE_F64, data=data, n_batch=2)
    ref2, _, _ = X.pne_open(net2, 8, E.LOOP)
    np.testing.assert_allclose(mant2[0] * math.exp(ls2[0]), ref, rtol=1e-10)
    np.testing.assert_allclose(mant2[1] * math.exp(ls2[1]), ref2, rtol=1e-10)


# ---------------------------------------------------------------- edge cases
def test_low_orders_and_trees(ctx):
    net = I.random_tensors(I.square_lattice(5, 4, 3), 2)
    ref0 = X.pne(net, 0, E.LOOP)
    for K in (0, 1, 2, 3):
        (r,) = ctx.expand(net, K, pne.PNE_MODE_LOOP, pne.PNE_F64)
        assert r["n_clusters"] == 0 and r["n_terms"] == 1
        assert abs(r["log_abs"] - ref0.log_abs) < 1e-10
    tree = I.random_tensors(I.grid_graph(6, [(0, 1), (1, 2), (1, 3), (3, 4), (4, 5)], [3, 2, 4, 2, 3]), 8)
    (r,) = ctx.expand(tree, 10, pne.PNE_MODE_LOOP, pne.PNE_F64)
    assert r["n_clusters"] == 0
    assert r["value"] == pytest.approx(float(Ex.contract_einsum(tree)), rel=1e-12)
    single = I.grid_graph(1, [], [])
    single = single.with_tensors([np.array(3.25)])
    (r,) = ctx.expand(single, 4, pne.PNE_MODE_LOOP, pne.PNE_F64)
    assert r["value"] == pytest.approx(3.25, rel=1e-15)


def test_multi_edges_and_irregular_graph(ctx):
    g = I.grid_graph(5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 2), (0, 1), (3, 1)], [2, 3, 2, 2, 3, 2, 2, 3])
    net = I.random_tensors(g, 4)
    # K = 1 and 2 reach the parallel pair (0, 1) exactly at the order limit
    for K in (1, 2, 3, 5, 8):
        ref = X.pne(net, K, E.LOOP)
        (res,), (edges, w) = ctx.expand(net, K, pne.PNE_MODE_LOOP, pne.PNE_F64, export=True)
        cl, wc = _canon(edges, w)
        assert cl == list(ref.clusters)
        np.testing.assert_allclose(wc[0], ref.w, rtol=1e-10, atol=1e-13)
        _check_values(res, ref)


def _random_multigraph(seed):
    # a connected random multigraph (parallel bonds allowed), site degree <= 6
    rng = np.random.default_rng(1000 + seed)
    n = 7 + seed % 4
    m = n + 5 + seed
    deg = np.zeros(n, dtype=int)
    edges = [(v, v + 1) for v in range(n - 1)]            # a path keeps it connected
    for a, b in edges:
        deg[a] += 1; deg[b] += 1
    while len(edges) < m:
        a, b = (int(x) for x in rng.integers(0, n, size=2))
        if a == b or deg[a] >= 6 or deg[b] >= 6:
            continue
        edges.append((min(a, b), max(a, b)))
        deg[a] += 1; deg[b] += 1
    dims = [int(d) for d in rng.integers(2, 4, size=m)]
    return I.grid_graph(n, edges, dims)


@pytest.mark.parametrize("seed", range(6))
def test_random_multigraph_clusters_and_values(ctx, seed):
    # the search's closing level (sizes K - 1 and K from the size K - 2 sets)
    # and its two-bond closing test, on irregular graphs with parallel bonds:
    # cluster lists bit-exact, values within the FP64 tolerance
    net = I.random_tensors(_random_multigraph(seed), seed)
    for K in (3, 4, 6, 8):
        ref = X.pne(net, K, E.LOOP)
        (res,), (edges, w) = ctx.expand(net, K, pne.PNE_MODE_LOOP, pne.PNE_F64, export=True)
        cl, wc = _canon(edges, w)
        assert cl == list(ref.clusters), (seed, K)
        np.testing.assert_allclose(wc[0], ref.w, rtol=1e-10, atol=1e-13)
        _check_values(res, ref)


def test_invalid_input_is_rejected(ctx):
    net = I.random_tensors(I.square_lattice(3, 3, 2), 1)
    bad = I.Network(net.n_sites, net.bond_site, np.full(net.n_bonds, 9, dtype=np.int32), net.site_ptr,
                    net.site_bonds, net.leg_dir, net.tensors)
    with pytest.raises(pne.PneError) as ei:
        ctx.expand(bad, 4, data=np.zeros(10 ** 5))
    assert ei.value.status == pne.PNE_EINVAL
    with pytest.raises(pne.PneError):
        ctx.expand(net, 40)           # order above the limit


def test_torch_allocator_gives_identical_results():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    net = I.random_tensors(I.square_lattice(6, 6, 3), 4)
    c1 = pne.Context(0)
    c2 = pne.Context(0, torch_alloc=True)
    try:
        (a,) = c1.expand(net, 8)
        (b,) = c2.expand(net, 8)
    finally:
        c1.close(); c2.close()
    assert np.array_equal(a["c"], b["c"])


# ---------------------------------------------------------------- float-float BP sweeps
FF_CASES = [
    ("random2d_D4", lambda: I.random_tensors(I.square_lattice(8, 8, 4), 3), 8),
    ("random2d_D5", lambda: I.random_tensors(I.square_lattice(6, 7, 5), 4), 6),
    ("random3d_D3", lambda: I.random_tensors(I.cubic_lattice(3, 3, 3, 3), 5, "n1,0.3"), 6),
    ("aklt", lambda: I.aklt_tensors(I.square_lattice(6, 6, 4)), 8),
    ("ising3d_ordered", lambda: I.ising_tensors(I.cubic_lattice(4, 4, 4, 2), 0.25), 8),
    ("ising2d", lambda: I.ising_tensors(I.square_lattice(4, 4, 2), 0.40), 24),
    ("bias_signed", lambda: I.random_tensors(I.square_lattice(5, 5, 3), 7, "bias:0.5"), 8),
    # dimension-4 sites (the half-warp pair form) beside sites with a
    # dimension-3 leg (the one-site form) in every colour class
    ("mixed_D34", lambda: _mixed_d34(), 6),
]


def _mixed_d34():
    g = I.square_lattice(7, 6, 4)
    g.bond_dim[::5] = 3
    return I.random_tensors(g, 12)


@pytest.mark.parametrize("name,make,K", FF_CASES, ids=[c[0] for c in FF_CASES])
def test_float_float_bp_matches_oracle(ctx, name, make, K):
    net = make()
    ref = X.pne(net, K, E.LOOP)
    (ff,) = ctx.expand(net, K, pne.PNE_MODE_LOOP, pne.PNE_F64, arithmetic=1)
    (d64,) = ctx.expand(net, K, pne.PNE_MODE_LOOP, pne.PNE_F64, arithmetic=0)
    assert ff["n_terms"] == ref.n_terms
    _check_values(ff, ref)
    assert abs(ff["log_abs"] - d64["log_abs"]) <= 1e-10
    assert ff["bp_iters"] > 0


@pytest.mark.parametrize("arith", [0, 1], ids=["fp64", "ff"])
@pytest.mark.parametrize("name", ["random2d_D4", "bias_signed", "mixed_D34"])
def test_damped_bp_reaches_the_same_fixed_point(ctx, name, arith):
    # damping changes the path to the fixed point, not the fixed point
    make, K = {c[0]: (c[1], c[2]) for c in FF_CASES}[name]
    net = make()
    ref = X.pne(net, K, E.LOOP)
    (r,) = ctx.expand(net, K, pne.PNE_MODE_LOOP, pne.PNE_F64, arithmetic=arith, damping=0.3)
    (u,) = ctx.expand(net, K, pne.PNE_MODE_LOOP, pne.PNE_F64, arithmetic=arith)
    _check_values(r, ref)
    assert r["bp_iters"] > u["bp_iters"] > 0


@pytest.mark.parametrize("cache", [0, 1])
@pytest.mark.parametrize("shape,D,K,mc,seed", [((6, 6), 3, 8, 4, 3), ((5, 5), 2, 10, 6, 4), ((4, 4), 4, 8, 8, 5)])
def test_cluster_size_cap_matches_the_oracle(ctx, shape, D, K, mc, seed, cache):
    # clusters of at most mc bonds, terms still up to order K built from them
    net = I.random_tensors(I.square_lattice(shape[0], shape[1], D), seed)
    cl = E.enumerate_clusters(net, mc, E.LOOP)
    ref = X.pne(net, K, E.LOOP, clusters=cl, terms=E.enumerate_terms(net, cl, K))
    (r,) = ctx.expand(net, K, pne.PNE_MODE_LOOP, pne.PNE_F64, max_cluster=mc, use_cache=bool(cache))
    assert r["n_clusters"] == len(cl) and r["n_terms"] == ref.n_terms
    _check_values(r, ref)
    if mc < K:
        (full,) = ctx.expand(net, K, pne.PNE_MODE_LOOP, pne.PNE_F64, use_cache=bool(cache))
        assert full["n_terms"] > r["n_terms"]       # a cached record of the other cap is not reused


# ---------------------------------------------------------------- search schedule
@pytest.mark.parametrize("shape,D,K,limit", [((8, 8), 3, 8, 1), ((8, 8), 3, 8, 700), ((8, 8), 3, 8, 6000),
                                             ((6, 5), 2, 10, 0), ((6, 5), 2, 10, 500)])
def test_search_arena_limit_gives_identical_lists(ctx, monkeypatch, shape, D, K, limit):
    """The breadth-first prefix stops where its node arena is full and the rest
    of the tree is searched depth-first (limit 1: depth-first from the anchors;
    limit 0: the default arena, and K = 10 ends depth-first from level 8).  The
    cluster list, its order and every value must not depend on where the
    search switches."""
    net = I.random_tensors(I.square_lattice(shape[0], shape[1], D), 5)
    (ref,), (e0, w0) = ctx.expand(net, K, pne.PNE_MODE_LOOP, pne.PNE_F64, export=True, use_cache=False)
    if limit:
        monkeypatch.setenv("PNE_SEARCH_ARENA_MAX", str(limit))
    c2 = pne.Context(0)
    monkeypatch.delenv("PNE_SEARCH_ARENA_MAX", raising=False)
    try:
        (res,), (e1, w1) = c2.expand(net, K, pne.PNE_MODE_LOOP, pne.PNE_F64, export=True, use_cache=False)
        # a second search on the same context starts from the arena size that fitted
        (res2,), (e2, _) = c2.expand(net, K, pne.PNE_MODE_LOOP, pne.PNE_F64, export=True, use_cache=False)
    finally:
        c2.close()
    assert np.array_equal(e0, e1) and np.array_equal(e0, e2)
    assert np.array_equal(w0, w1)
    assert res["n_terms"] == ref["n_terms"] == res2["n_terms"]
    assert res["log_abs"] == ref["log_abs"]
    if K == 10:
        refo = X.pne(net, K, E.LOOP)
        cl, _ = _canon(e1, None)
        assert cl == list(refo.clusters)
        _check_values(res, refo)


# ---------------------------------------------------------------- deferred BP record, two streams
def test_async_partition_and_enumeration_on_a_second_stream(ctx):
    """The partition built without waiting for its BP record, the enumeration
    run on another stream (it waits for the geometry only), the contraction
    joined back: the same values bit for bit as the plain synchronous flow,
    with the convergence record read by pne_sum."""
    g = I.square_lattice(8, 8, 4)
    nets = [I.random_tensors(g, s) for s in (11, 12)]
    flat = np.concatenate([n.flat_data()[0] for n in nets])
    data = torch.from_numpy(flat).cuda()
    K = 8
    ns, keep = pne.network_struct(g, data=data, n_batch=2)
    part, _ = pne.pne_build_partition(ctx.h, ns, pne.PartitionOpts(1e-13, 10000, 0.0, 1, 0), None)
    terms, _, _ = pne.pne_enumerate_terms(ctx.h, part, pne.EnumOpts(K, pne.PNE_MODE_LOOP, 0), None)
    pne.pne_contract_terms(ctx.h, terms, pne.PNE_F64, None)
    ref = pne.pne_sum(ctx.h, terms, None)
    pne.pne_terms_destroy(terms); pne.pne_partition_destroy(part)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ev = torch.cuda.Event()
    for _ in range(2):
        part, _ = pne.pne_build_partition(ctx.h, ns, pne.PartitionOpts(1e-13, 10000, 0.0, 1, 1), s1.cuda_stream)
        terms, _, _ = pne.pne_enumerate_terms(ctx.h, part, pne.EnumOpts(K, pne.PNE_MODE_LOOP, 0), s2.cuda_stream)
        ev.record(s2)
        s1.wait_event(ev)
        pne.pne_contract_terms(ctx.h, terms, pne.PNE_F64, s1.cuda_stream)
        got = pne.pne_sum(ctx.h, terms, s1.cuda_stream)
        pne.pne_terms_destroy(terms); pne.pne_partition_destroy(part)
        for a, b in zip(got, ref):
            assert a["log_abs"] == b["log_abs"] and a["sign"] == b["sign"]
            assert np.array_equal(a["c"], b["c"])
            assert a["bp_iters"] == b["bp_iters"] > 0
    torch.cuda.synchronize()
    del keep
    # a deferred record that shows non-convergence: pne_sum reports it after
    # writing the results
    part, _ = pne.pne_build_partition(ctx.h, ns, pne.PartitionOpts(1e-13, 2, 0.0, 1, 1), None)
    terms, _, _ = pne.pne_enumerate_terms(ctx.h, part, pne.EnumOpts(4, pne.PNE_MODE_LOOP, 0), None)
    pne.pne_contract_terms(ctx.h, terms, pne.PNE_F64, None)
    with pytest.raises(pne.PneError) as ei:
        pne.pne_sum(ctx.h, terms, None)
    assert ei.value.status == pne.PNE_ENOCONV
    res = pne.pne_sum(ctx.h, terms, None, allow_noconv=True)
    assert all(r["bp_iters"] == 0 for r in res)
    pne.pne_terms_destroy(terms); pne.pne_partition_destroy(part)


def test_full_size_cluster_and_term_counts_match_the_oracle_golden_file(ctx):
    # lattices too large for the oracle inside a test run (the 16x16 bench
    # geometry and the 8x8x8 one among them): counts written by the oracle
    # (tests/golden/make_golden.py), bit-exact on the GPU, clusters by size too
    import json
    import os
    from collections import Counter
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cluster_counts.json")))["cases"]
    geoms = {"square16x16": I.square_lattice(16, 16, 2), "square24x24": I.square_lattice(24, 24, 2),
             "cubic6x6x6": I.cubic_lattice(6, 6, 6, 2), "cubic8x8x8": I.cubic_lattice(8, 8, 8, 2),
             "cubic4x4x4_K10": I.cubic_lattice(4, 4, 4, 2), "cubic8x8x8_K10": I.cubic_lattice(8, 8, 8, 2)}
    assert set(geoms) == set(golden)
    for name, g in geoms.items():
        ref = golden[name]
        net = I.ising_tensors(g, 0.3)
        ns, keep = pne.network_struct(net)
        part, _ = pne.pne_build_partition(ctx.h, ns, pne.PartitionOpts(1e-13, 10000, 0.0))
        try:
            terms, nc, nt = pne.pne_enumerate_terms(ctx.h, part, pne.EnumOpts(ref["K"], pne.PNE_MODE_LOOP, 0))
            try:
                assert (nc, nt) == (ref["n_clusters"], ref["n_terms"]), name
                edges, _ = pne.pne_terms_export(ctx.h, terms, nc, ref["K"], with_values=False)
                by_size = Counter(int((row >= 0).sum()) for row in edges)
                assert {str(k): v for k, v in sorted(by_size.items())} == ref["clusters_by_size"], name
            finally:
                pne.pne_terms_destroy(terms)
        finally:
            pne.pne_partition_destroy(part)
        del keep


@pytest.mark.parametrize("K", [8, 10])
def test_ising_8x8x8_values_match_the_high_temperature_closed_form(ctx, K):
    # 3D Ising 8x8x8 at orders 8 and 10 (the full-size cubic workload): in the
    # paramagnetic gauge a cluster's weight is tanh(beta)^|C| when every vertex
    # has even degree and 0 otherwise, so c_k = n_k tanh(beta)^k with n_k the
    # even subgraphs of k bonds, counted by the oracle (golden file), and
    # Z_BP = 2^N cosh(beta)^M.  FP64 values within 1e-10; TF32 and BF16 within
    # their stated bounds.
    import json
    import os
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cluster_counts.json")))["cases"]
    even = {int(k): v for k, v in golden["cubic8x8x8_K10"]["even_terms_by_order"].items()}
    g = I.cubic_lattice(8, 8, 8, 2)
    betas = (0.20, 0.2217, 0.25)
    nets = [I.ising_tensors(g, b) for b in betas]
    data = np.concatenate([n.flat_data()[0] for n in nets])
    for dtype in ("f64", "tf32", "bf16"):
        res = ctx.expand(nets[0], K, pne.PNE_MODE_LOOP, dtype, data=data, n_batch=len(nets))
        for r, b in zip(res, betas):
            t = math.tanh(b)
            ck = np.array([even.get(k, 0) * t ** k for k in range(K + 1)])
            lz = g.n_sites * math.log(2.0) + g.n_bonds * math.log(math.cosh(b)) + math.log(ck.sum())
            rel = abs(math.expm1(r["log_abs"] - lz))
            if dtype == "f64":
                assert rel <= 1e-10, (b, rel)
                np.testing.assert_allclose(r["c"], ck, rtol=0, atol=1e-12 * ck.sum())
            else:
                assert rel <= r["err_bound"] <= BOUND_CAP[dtype], (dtype, b, rel, r["err_bound"])

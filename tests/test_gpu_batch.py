"""Batched form: one persistent fused launch over many networks (uneven sizes
and bond dimensions), replayed from a CUDA graph, against the per-network
path and the oracle."""
import numpy as np
import pytest

from paper_2512_10910_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2512_10910_gb300 import pne  # noqa: E402
from oracle import enumerate as E  # noqa: E402
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


def _groups():
    """(geometry, list of networks) groups of several sizes and dimensions."""
    out = []
    for (L, D, seeds) in [(6, 2, (1, 2)), (7, 3, (3,)), (5, 4, (4, 5, 6)), (8, 5, (7,)), (6, 6, (8,))]:
        g = I.square_lattice(L, L, D)
        out.append((g, [I.random_tensors(g, s) for s in seeds]))
    g = I.square_lattice(7, 6, 2)
    out.append((g, [I.ising_tensors(g, b) for b in (0.3, 0.45)]))
    return out


def _make(ctx, groups, K=8):
    parts, terms, keep = [], [], []
    for g, nets in groups:
        data = np.concatenate([n.flat_data()[0] for n in nets])
        ns, kp = pne.network_struct(g, data=data, n_batch=len(nets))
        p, _ = pne.pne_build_partition(ctx.h, ns, pne.PartitionOpts(1e-13, 10000, 0.0))
        t, _, _ = pne.pne_enumerate_terms(ctx.h, p, pne.EnumOpts(K, 0, 1))
        parts.append(p); terms.append(t); keep.append((ns, kp))
    return parts, terms, keep


def _free(parts, terms):
    for t in terms:
        pne.pne_terms_destroy(t)
    for p in parts:
        pne.pne_partition_destroy(p)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_matches_per_network_path_and_oracle(ctx, dtype):
    groups = _groups()
    parts, terms, keep = _make(ctx, groups)
    try:
        b = pne.pne_batch_create(ctx.h, terms, pne.DTYPES[dtype])
        got = pne.pne_batch_run(ctx.h, b)
        w, k, ms = pne.pne_batch_config(b)
        assert w in (1, 2, 4, 8) and k >= 1 and ms > 0
        assert pne.pne_batch_schedule(b) in (pne.PNE_SCHED_HANDLE, pne.PNE_SCHED_LARGEST_FIRST)
        pne.pne_batch_destroy(b)
        r = 0
        for (g, nets), t in zip(groups, terms):
            pne.pne_contract_terms(ctx.h, t, pne.DTYPES[dtype])
            single = pne.pne_sum(ctx.h, t)
            for j, net in enumerate(nets):
                one, ref = got[r], single[j]
                assert one["n_terms"] == ref["n_terms"] and one["n_clusters"] == ref["n_clusters"]
                tol = 1e-12 if dtype == "f64" else 1e-6
                assert abs(one["log_abs"] - ref["log_abs"]) <= tol
                np.testing.assert_allclose(one["c"], ref["c"], rtol=0, atol=tol * np.sum(np.abs(ref["c"])))
                if dtype == "f64":
                    orc = X.pne(net, 8, E.LOOP)
                    assert abs(one["log_abs"] - orc.log_abs) <= 1e-10
                r += 1
        assert r == len(got)
    finally:
        _free(parts, terms)


def test_batch_results_identical_across_launch_shapes_and_graph(ctx):
    groups = _groups()
    parts, terms, keep = _make(ctx, groups)
    try:
        runs = []
        for opts in (pne.BatchOpts(1, 1, 1), pne.BatchOpts(2, 1, 1), pne.BatchOpts(1, 2, 0), None,
                     pne.BatchOpts(2, 1, 1, pne.PNE_SCHED_LARGEST_FIRST),
                     pne.BatchOpts(1, 2, 0, pne.PNE_SCHED_LARGEST_FIRST)):
            b = pne.pne_batch_create(ctx.h, terms, pne.PNE_F64, opts)
            if opts is not None:
                assert pne.pne_batch_schedule(b) == opts.schedule
            runs.append([(r["log_abs"], tuple(r["c"])) for r in pne.pne_batch_run(ctx.h, b)])
            runs.append([(r["log_abs"], tuple(r["c"])) for r in pne.pne_batch_run(ctx.h, b)])   # replay
            pne.pne_batch_destroy(b)
        for other in runs[1:]:
            assert other == runs[0]
    finally:
        _free(parts, terms)


def test_batch_rejects_a_shape_that_does_not_fit(ctx):
    groups = _groups()
    parts, terms, keep = _make(ctx, groups)
    try:
        with pytest.raises(pne.PneError) as ei:
            pne.pne_batch_create(ctx.h, terms, pne.PNE_F64, pne.BatchOpts(32, 8, 1))
        assert ei.value.status == pne.PNE_EINVAL
        with pytest.raises(pne.PneError) as ei:
            pne.pne_batch_create(ctx.h, terms, pne.PNE_F64, pne.BatchOpts(1, 1, 1, 7))
        assert ei.value.status == pne.PNE_EINVAL
    finally:
        _free(parts, terms)


def test_batch_after_partition_update(ctx):
    g = I.square_lattice(6, 6, 3)
    nets_a = [I.random_tensors(g, s) for s in (1, 2)]
    nets_b = [I.random_tensors(g, s) for s in (3, 4)]
    parts, terms, keep = _make(ctx, [(g, nets_a)])
    try:
        b = pne.pne_batch_create(ctx.h, terms, pne.PNE_F64)
        pne.pne_batch_run(ctx.h, b)
        data = torch.from_numpy(np.concatenate([n.flat_data()[0] for n in nets_b])).cuda()
        pne.pne_partition_update(ctx.h, parts[0], data)
        got = pne.pne_batch_run(ctx.h, b)
        pne.pne_batch_destroy(b)
        for r, net in zip(got, nets_b):
            (fresh,) = ctx.expand(net, 8)
            assert abs(r["log_abs"] - fresh["log_abs"]) <= 1e-12
    finally:
        _free(parts, terms)


def test_batch_after_asynchronous_updates_on_two_streams(ctx):
    # partition updates that defer their convergence record, issued on two
    # streams and joined into the batch's stream, give the same results, bit
    # for bit, as synchronous updates
    groups = [(I.square_lattice(6, 6, 3), [I.random_tensors(I.square_lattice(6, 6, 3), s) for s in (1, 2)]),
              (I.square_lattice(5, 7, 2), [I.ising_tensors(I.square_lattice(5, 7, 2), b) for b in (0.3, 0.4)])]
    parts, terms, keep = _make(ctx, groups)
    new = [torch.from_numpy(np.concatenate([I.random_tensors(groups[0][0], s).flat_data()[0] for s in (5, 6)])).cuda(),
           torch.from_numpy(np.concatenate([I.ising_tensors(groups[1][0], b).flat_data()[0] for b in (0.35, 0.45)])).cuda()]
    try:
        b = pne.pne_batch_create(ctx.h, terms, pne.PNE_F64)
        for p, d in zip(parts, new):
            pne.pne_partition_update(ctx.h, p, d)
        ref = [(r["log_abs"], tuple(r["c"]), r["bp_iters"]) for r in pne.pne_batch_run(ctx.h, b)]
        main = torch.cuda.current_stream()
        side = [torch.cuda.Stream(), torch.cuda.Stream()]
        for _ in range(2):
            for p, d, st in zip(parts, new, side):
                st.wait_stream(main)
                pne.pne_partition_update(ctx.h, p, d, pne.PartitionOpts(1e-13, 10000, 0.0, 0, 1), st.cuda_stream)
            for st in side:
                main.wait_stream(st)
            got = [(r["log_abs"], tuple(r["c"]), r["bp_iters"]) for r in pne.pne_batch_run(ctx.h, b)]
            assert got == ref
            assert all(it > 0 for _, _, it in got)
        pne.pne_batch_destroy(b)
    finally:
        _free(parts, terms)


def test_full_size_batch_members_match_the_oracle(ctx):
    # members of the 4096-network batch at its largest size (L = 24): a random
    # network at the largest bond dimension (D = 6) and an Ising network,
    # contracted by the fused batch kernel together with a small group,
    # against the FP64 oracle (the same draws as the batched workload)
    items = I.batched_workload_items([61, 171])
    assert [(k, L, D) for k, L, D, _, _ in items] == [("random", 24, 6), ("ising", 24, 2)]
    groups = [(net, [net]) for _, _, _, _, net in items] + _groups()[:1]
    parts, terms, keep = _make(ctx, groups)
    try:
        b = pne.pne_batch_create(ctx.h, terms, pne.PNE_F64, pne.BatchOpts(4, 2, 1))
        try:
            res = pne.pne_batch_run(ctx.h, b)
        finally:
            pne.pne_batch_destroy(b)
        for (_, _, _, _, net), r in zip(items, res[:2]):
            ref = X.pne(net, 8, E.LOOP)
            assert r["n_clusters"] == ref.n_clusters and r["n_terms"] == ref.n_terms
            assert abs(r["log_abs"] - ref.log_abs) <= 1e-10, (r["log_abs"], ref.log_abs)
            scale = float(np.sum(np.abs(ref.c)))
            np.testing.assert_allclose(r["c"], ref.c, rtol=0, atol=1e-10 * scale)
    finally:
        _free(parts, terms)


def test_batch_of_capped_enumerations_matches_the_oracle(ctx):
    # handles whose clusters are capped below the order (max_cluster) batch
    # like any other: terms of order <= K built from clusters of <= 4 bonds
    groups = [(I.square_lattice(6, 6, 3), [I.random_tensors(I.square_lattice(6, 6, 3), s) for s in (81, 82)]),
              (I.square_lattice(5, 5, 2), [I.random_tensors(I.square_lattice(5, 5, 2), 83)])]
    parts, terms, keep = [], [], []
    try:
        for g, nets in groups:
            data = np.concatenate([n.flat_data()[0] for n in nets])
            ns, kp = pne.network_struct(g, data=data, n_batch=len(nets))
            p, _ = pne.pne_build_partition(ctx.h, ns, pne.PartitionOpts(1e-13, 10000, 0.0))
            t, _, _ = pne.pne_enumerate_terms(ctx.h, p, pne.EnumOpts(8, 0, 1, 4))
            parts.append(p); terms.append(t); keep.append((ns, kp))
        b = pne.pne_batch_create(ctx.h, terms, pne.PNE_F64)
        got = pne.pne_batch_run(ctx.h, b)
        pne.pne_batch_destroy(b)
        r = 0
        for g, nets in groups:
            for net in nets:
                cl = E.enumerate_clusters(net, 4, E.LOOP)
                ref = X.pne(net, 8, E.LOOP, clusters=cl, terms=E.enumerate_terms(net, cl, 8))
                assert got[r]["n_terms"] == ref.n_terms
                assert abs(got[r]["log_abs"] - ref.log_abs) <= 1e-10
                np.testing.assert_allclose(got[r]["c"], ref.c, rtol=0, atol=1e-10 * np.sum(np.abs(ref.c)))
                r += 1
    finally:
        _free(parts, terms)

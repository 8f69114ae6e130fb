"""Per-kernel timing and the timeline: event-timed kernel records on the
streams they ran on, host stretches of library code, and identical results
with and without them."""
import time

import numpy as np
import pytest

from paper_2512_10910_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2512_10910_gb300 import pne  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2512_10910_gb300 import build
    build.build()
    c = pne.Context(0)
    yield c
    c.close()


def _run(ctx, g, nets, side=None):
    data = np.concatenate([n.flat_data()[0] for n in nets])
    ns, keep = pne.network_struct(g, data=data, n_batch=len(nets))
    p, _ = pne.pne_build_partition(ctx.h, ns, pne.PartitionOpts(1e-13, 10000, 0.0))
    try:
        t, _, _ = pne.pne_enumerate_terms(ctx.h, p, pne.EnumOpts(6, 0, 0), side)
        if side is not None:
            torch.cuda.synchronize()
        try:
            pne.pne_contract_terms(ctx.h, t, pne.PNE_F64)
            return [(r["log_abs"], tuple(r["c"])) for r in pne.pne_sum(ctx.h, t)]
        finally:
            pne.pne_terms_destroy(t)
    finally:
        pne.pne_partition_destroy(p)


def test_timeline_orders_kernels_and_host_stretches(ctx):
    g = I.square_lattice(6, 6, 3)
    nets = [I.random_tensors(g, s) for s in (1, 2)]
    plain = _run(ctx, g, nets)
    side = torch.cuda.Stream()
    t_before = time.monotonic() * 1000.0
    pne.pne_ctx_profile(ctx.h, True, trace=True)
    traced = _run(ctx, g, nets, side.cuda_stream)
    tr, origin = pne.pne_ctx_trace_read(ctx.h)
    sums = pne.pne_ctx_profile_read(ctx.h)
    pne.pne_ctx_profile(ctx.h, False)
    assert traced == plain
    assert origin >= t_before
    gpu = [e for e in tr if e["kind"] == "gpu"]
    host = [e for e in tr if e["kind"] == "host"]
    assert gpu and host
    assert all(e["t1_ms"] >= e["t0_ms"] >= 0.0 for e in tr)
    assert [e["t0_ms"] for e in tr] == sorted(e["t0_ms"] for e in tr)
    # the partition's stream comes first, the enumeration's second (the
    # contraction may fork further side streams)
    assert gpu[0]["stream"] == 0 and {0, 1} <= {e["stream"] for e in gpu}
    assert all(e["stream"] == -1 for e in host)
    # every kernel family of the sums appears in the timeline, as often
    names = [e["name"] for e in gpu]
    for fam, (launches, total) in sums.items():
        if fam.startswith("host:"):
            assert sum(1 for e in host if e["name"] == fam[5:]) == launches
        else:
            assert names.count(fam) == launches
            assert abs(sum(e["t1_ms"] - e["t0_ms"] for e in gpu if e["name"] == fam) - total) <= 1e-6 * max(1.0, total)


def test_trace_off_records_nothing(ctx):
    pne.pne_ctx_profile(ctx.h, True)
    g = I.square_lattice(4, 4, 2)
    _run(ctx, g, [I.random_tensors(g, 3)])
    tr, _ = pne.pne_ctx_trace_read(ctx.h)
    pne.pne_ctx_profile(ctx.h, False)
    assert tr == []

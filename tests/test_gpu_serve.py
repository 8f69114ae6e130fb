"""Served form: continuous batching with memory admission.  Each request's
result is the same alone and inside a mix of concurrent requests, and equals
the single-request path."""
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


def _requests():
    reqs = []
    for L, K in ((6, 6), (8, 8), (5, 4), (9, 8)):
        reqs.append((I.aklt_tensors(I.square_lattice(L, L, 4)), K))
    for L, D, K, sd in ((3, 2, 8, 1), (4, 3, 6, 2), (3, 4, 8, 3), (5, 2, 4, 4)):
        reqs.append((I.random_tensors(I.cubic_lattice(L, L, L, D), sd, "n1,0.3"), K))
    return reqs


def _wait(srv, rid, timeout=120.0):
    t0 = time.time()
    while True:
        st, res, info = pne.pne_server_poll(srv, rid)
        if st != pne.PNE_EBUSY:
            assert st == pne.PNE_OK, st
            return res, info
        assert time.time() - t0 < timeout
        time.sleep(0.001)


@pytest.mark.parametrize("dtype", [pne.PNE_F64, pne.PNE_F32])
def test_alone_equals_in_mix_and_single_path(ctx, dtype):
    reqs = _requests()
    structs = [pne.network_struct(net) for net, _ in reqs]
    srv = pne.pne_server_create(ctx.h, pne.ServerOpts(0, 0, 3, 0, dtype, 0, 0))
    try:
        alone = []
        for (net, K), (ns, _) in zip(reqs, structs):
            rid = pne.pne_server_submit(srv, ns, K)
            res, info = _wait(srv, rid)
            assert info["batch_size"] == 1
            alone.append(res)
        ids = [pne.pne_server_submit(srv, ns, K) for (net, K), (ns, _) in zip(reqs, structs)]
        mix = [_wait(srv, rid) for rid in ids]
        assert max(info["batch_size"] for _, info in mix) > 1        # they did share launches
        for a, (m, info) in zip(alone, mix):
            assert a["log_abs"] == m["log_abs"] and np.array_equal(a["c"], m["c"])
            assert info["t_arrival"] <= info["t_admit"] <= info["t_ready"] <= info["t_done"]
    finally:
        pne.pne_server_destroy(srv)
    for (net, K), a in zip(reqs, alone):
        (single,) = ctx.expand(net, K, pne.PNE_MODE_LOOP, dtype, arithmetic=1)   # the server's BP arithmetic
        tol = 1e-12 if dtype == pne.PNE_F64 else 1e-6
        assert abs(single["log_abs"] - a["log_abs"]) <= tol
        assert single["n_terms"] == a["n_terms"]


def test_admission_respects_the_budget(ctx):
    reqs = _requests() * 2
    structs = [pne.network_struct(net) for net, _ in reqs]
    budget = 4 << 20
    srv = pne.pne_server_create(ctx.h, pne.ServerOpts(budget, 0, 4, 0, pne.PNE_F32, 0, 0))
    try:
        ids = [pne.pne_server_submit(srv, ns, K) for (net, K), (ns, _) in zip(reqs, structs)]
        out = [_wait(srv, rid) for rid in ids]
        peak, _ = pne.pne_server_stats(srv)
        biggest = max(info["device_bytes"] for _, info in out)
        assert peak <= max(budget, biggest)
        assert all(r["n_terms"] > 0 for r, _ in out)
    finally:
        pne.pne_server_destroy(srv)


def test_failed_request_reports_its_status_and_error_text(ctx):
    # a network whose tensors are all zero has zero BP messages: the partition
    # reports PNE_EDEGENERATE (a flag the kernels set, no fault); the server
    # finishes that request with the status, keeps serving the others, and
    # records the failing call's message
    good = I.aklt_tensors(I.square_lattice(5, 5, 4))
    bad = I.aklt_tensors(I.square_lattice(5, 5, 4))
    flat = np.zeros_like(bad.flat_data()[0])
    ns_bad, keep_bad = pne.network_struct(bad, data=flat)
    ns_good, keep_good = pne.network_struct(good)
    srv = pne.pne_server_create(ctx.h, pne.ServerOpts(0, 0, 2, 0, pne.PNE_F64, 0, 0))
    try:
        assert pne.pne_server_first_error(srv) == ""
        rid_bad = pne.pne_server_submit(srv, ns_bad, 4)
        rid_good = pne.pne_server_submit(srv, ns_good, 4)
        pne.pne_server_drain(srv)
        st, res, info = pne.pne_server_poll(srv, rid_bad)
        assert st == pne.PNE_EDEGENERATE and res is None
        res, info = _wait(srv, rid_good)
        assert res["n_terms"] > 0
        msg = pne.pne_server_first_error(srv)
        assert msg.startswith("request %d:" % rid_bad) and "zero message" in msg
    finally:
        pne.pne_server_destroy(srv)

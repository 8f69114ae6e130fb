"""User projectors instead of BP (pne_partition_opts.use_user_projectors), through
the C ABI, against the FP64 oracle given the same projectors.

Eq. A2-A4 hold for any complementary P, Q: with every term kept (ALL mode, full
order) the expansion equals the exact contraction whatever the projectors; in
LOOP mode, away from a BP fixed point, the dangling terms no longer vanish, so
the GPU is compared with the oracle's LOOP expansion on the same projectors
(cluster values and per-order sums within 1e-10 of sum |c_k|).  The BP fixed
point passed as user projectors reproduces the BP path; a zero overlap is
PNE_EDEGENERATE.
"""
import math

import numpy as np
import pytest

from paper_2512_10910_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2512_10910_gb300 import pne  # noqa: E402
from oracle import bp as Bp  # noqa: E402
from oracle import enumerate as E  # noqa: E402
from oracle import exact as X  # noqa: E402
from oracle import expansion as Ex  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2512_10910_gb300 import build
    build.build()
    c = pne.Context(0)
    yield c
    c.close()


def _closed(net):
    return [b for b in range(net.n_bonds) if int(net.bond_site[b][1]) >= 0]


def _random_vectors(net, seed, spread=0.5):
    """u_b, v_b per closed bond: 1 + U[-spread, spread] entries (overlaps far from 0)."""
    rng = np.random.default_rng(seed)
    uv = {}
    for b in _closed(net):
        d = int(net.bond_dim[b])
        uv[b] = (1.0 + rng.uniform(-spread, spread, d), 1.0 + rng.uniform(-spread, spread, d))
    return uv


def _flat(net, uvs):
    """[sets][closed bonds in id order][bond_dim[b]] for u and for v."""
    u = np.concatenate([np.concatenate([uv[b][0] for b in _closed(net)]) for uv in uvs])
    v = np.concatenate([np.concatenate([uv[b][1] for b in _closed(net)]) for uv in uvs])
    return u, v


def _oracle_proj(net, uv):
    """The oracle's (P, Q, cap0, cap1) per bond for P_b = u v^T / (u . v)."""
    proj = []
    for b in range(net.n_bonds):
        if int(net.bond_site[b][1]) < 0:
            proj.append(None)
            continue
        u, v = uv[b]
        cap0, cap1 = u.copy(), v / float(u @ v)
        P = np.outer(cap0, cap1)
        proj.append((P, np.eye(len(u)) - P, cap0, cap1))
    return proj


def _check(res, ref, tol=1e-10):
    assert res["sign"] == ref.sign
    assert abs(res["log_abs"] - ref.log_abs) <= tol * max(1.0, abs(ref.log_abs)), (res["log_abs"], ref.log_abs)
    scale = float(np.sum(np.abs(ref.c)))
    np.testing.assert_allclose(res["c"], ref.c, rtol=0, atol=tol * scale)


def test_all_mode_full_order_is_exact_for_any_projectors(ctx):
    # every P/Q string kept: Eq. A3-A4 reproduce the network exactly
    net = I.random_tensors(I.square_lattice(3, 3, 2), 21)
    uv = _random_vectors(net, 5)
    K = len(_closed(net))
    (r,) = ctx.expand(net, K, pne.PNE_MODE_ALL, pne.PNE_F64, projectors=_flat(net, [uv]))
    t, ls = X.contract_sweep(net)
    exact = math.log(abs(float(t))) + ls
    assert abs(r["log_abs"] - exact) < 1e-12 * abs(exact)
    assert r["bp_iters"] == 0
    _check(r, Ex.pne(net, K, E.ALL, proj=_oracle_proj(net, uv)))


@pytest.mark.parametrize("arith", [0, 1], ids=["fp64", "ff"])
@pytest.mark.parametrize("shape,D,K,seed", [((6, 5), 3, 8, 1), ((5, 4), 4, 6, 2), ((3, 3), 2, 8, 3)])
def test_loop_mode_matches_the_oracle_on_the_same_projectors(ctx, shape, D, K, seed, arith):
    net = I.random_tensors(I.square_lattice(shape[0], shape[1], D), seed)
    uv = _random_vectors(net, 100 + seed)
    (r,) = ctx.expand(net, K, pne.PNE_MODE_LOOP, pne.PNE_F64, projectors=_flat(net, [uv]), arithmetic=arith)
    ref = Ex.pne(net, K, E.LOOP, proj=_oracle_proj(net, uv))
    assert r["n_terms"] == ref.n_terms
    _check(r, ref)


def test_each_tensor_set_takes_its_own_projectors(ctx):
    g = I.square_lattice(4, 3, 3)
    nets = [I.random_tensors(g, 40 + i) for i in range(2)]
    uvs = [_random_vectors(nets[i], 60 + i) for i in range(2)]
    flat = np.concatenate([n.flat_data()[0] for n in nets])
    res = ctx.expand(g, 6, pne.PNE_MODE_LOOP, pne.PNE_F64, data=flat, n_batch=2, projectors=_flat(g, uvs))
    for r, net, uv in zip(res, nets, uvs):
        _check(r, Ex.pne(net, 6, E.LOOP, proj=_oracle_proj(net, uv)))


def test_the_bp_fixed_point_as_user_projectors_reproduces_the_bp_path(ctx):
    net = I.random_tensors(I.square_lattice(5, 5, 3), 9)
    bpres = Bp.bp_fixed_point(net)
    proj = Bp.bond_projectors(net, bpres)
    uv = {b: (proj[b][2], proj[b][3]) for b in _closed(net)}      # P = cap0 cap1^T, cap0 . cap1 = 1
    (user,) = ctx.expand(net, 8, pne.PNE_MODE_LOOP, pne.PNE_F64, projectors=_flat(net, [uv]))
    (bp,) = ctx.expand(net, 8, pne.PNE_MODE_LOOP, pne.PNE_F64)
    assert user["n_terms"] == bp["n_terms"]
    assert abs(user["log_abs"] - bp["log_abs"]) < 1e-10
    np.testing.assert_allclose(user["c"], bp["c"], rtol=0, atol=1e-10 * float(np.sum(np.abs(bp["c"]))))


def test_orthogonal_projector_vectors_are_degenerate(ctx):
    net = I.random_tensors(I.square_lattice(3, 3, 2), 4)
    uv = _random_vectors(net, 8)
    b0 = _closed(net)[3]
    uv[b0] = (np.array([1.0, 0.0]), np.array([0.0, 1.0]))            # u . v = 0
    with pytest.raises(pne.PneError) as e:
        ctx.expand(net, 6, pne.PNE_MODE_LOOP, pne.PNE_F64, projectors=_flat(net, [uv]))
    assert e.value.status == pne.PNE_EDEGENERATE


def test_partition_update_with_user_projectors(ctx):
    # the handle built by BP, then updated in place with new tensors and user
    # projectors: the enumeration built on it stays valid and the sums follow
    # the new projectors
    g = I.square_lattice(4, 4, 3)
    net0, net1 = I.random_tensors(g, 71), I.random_tensors(g, 72)
    ns, keep = pne.network_struct(net0)
    part, _ = pne.pne_build_partition(ctx.h, ns, pne.PartitionOpts(1e-13, 10000, 0.0))
    try:
        terms, _, _ = pne.pne_enumerate_terms(ctx.h, part, pne.EnumOpts(6, pne.PNE_MODE_LOOP, 0))
        try:
            uv = _random_vectors(net1, 73)
            opts, pkeep = pne.user_projector_opts(*_flat(net1, [uv]))
            pne.pne_partition_update(ctx.h, part, net1.flat_data()[0], opts)
            pne.pne_contract_terms(ctx.h, terms, pne.PNE_F64)
            (r,) = pne.pne_sum(ctx.h, terms)
            _check(r, Ex.pne(net1, 6, E.LOOP, proj=_oracle_proj(net1, uv)))
            assert r["bp_iters"] == 0
            # and back to BP on the same handle
            pne.pne_partition_update(ctx.h, part, net1.flat_data()[0], pne.PartitionOpts(1e-13, 10000, 0.0))
            pne.pne_contract_terms(ctx.h, terms, pne.PNE_F64)
            (b,) = pne.pne_sum(ctx.h, terms)
            _check(b, Ex.pne(net1, 6, E.LOOP))
            assert b["bp_iters"] > 0
            del pkeep
        finally:
            pne.pne_terms_destroy(terms)
    finally:
        pne.pne_partition_destroy(part)


def test_user_projectors_with_a_deferred_record(ctx):
    # async_status: the record (zero sweeps, the gauge's degenerate flag) is read
    # by pne_sum; a good set of projectors sums normally, a zero overlap raises there
    net = I.random_tensors(I.square_lattice(4, 4, 2), 91)
    for degenerate in (False, True):
        uv = _random_vectors(net, 92)
        if degenerate:
            uv[_closed(net)[2]] = (np.array([1.0, 0.0]), np.array([0.0, 1.0]))
        opts, pkeep = pne.user_projector_opts(*_flat(net, [uv]), async_status=1)
        ns, keep = pne.network_struct(net)
        part, _ = pne.pne_build_partition(ctx.h, ns, opts)
        try:
            terms, _, _ = pne.pne_enumerate_terms(ctx.h, part, pne.EnumOpts(8, pne.PNE_MODE_LOOP, 0))
            try:
                pne.pne_contract_terms(ctx.h, terms, pne.PNE_F64)
                if degenerate:
                    with pytest.raises(pne.PneError) as e:
                        pne.pne_sum(ctx.h, terms)
                    assert e.value.status == pne.PNE_EDEGENERATE
                else:
                    (r,) = pne.pne_sum(ctx.h, terms)
                    _check(r, Ex.pne(net, 8, E.LOOP, proj=_oracle_proj(net, uv)))
                    assert r["bp_iters"] == 0
            finally:
                pne.pne_terms_destroy(terms)
        finally:
            pne.pne_partition_destroy(part)
        del pkeep

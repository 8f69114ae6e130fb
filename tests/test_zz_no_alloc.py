"""The allocation-free BP entry point, pne_bp_messages_noalloc.

Some callers must not allocate device memory while they run: a host framework
that has reserved the device's memory for its own allocator and lends the
library only fixed buffers, or a latency-critical loop where cudaMalloc and
cudaFree (and the synchronisation they can imply) are not allowed.  For them
the library offers BP to a fixed point whose working memory is a static device
array.  This test calls it twice in a row through the C ABI (the second call
reuses the array the first one left behind) and checks each result against the
regular path: the vacuum value ln|Z_BP| that pne_build_partition yields
(K = 0), within the 1e-10 FP64 tolerance of the other GPU tests, and the
oracle's fixed-point messages.  Around the second call the device's free
memory must not change (the first call may still load the library's device
code).  A network too large for the array is rejected before any GPU work.
The file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import math

import numpy as np
import pytest

from paper_2512_10910_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ln_zbp_from_messages(net, msg, B):
    """ln|Z_BP| from outgoing messages: every site capped by the messages
    arriving on its legs, divided by each bond's message overlap."""
    L = int(net.site_ptr[-1])
    m = msg.reshape(B, L, 8)
    slot = {}
    for v in range(net.n_sites):
        for k in range(net.site_ptr[v], net.site_ptr[v + 1]):
            slot[(v, int(net.site_bonds[k]))] = k
    out = []
    for b in range(B):
        lz = 0.0
        for v in range(net.n_sites):
            t = np.asarray(net._sets[b][v])
            legs = [int(x) for x in net.legs(v)]
            for i in reversed(range(len(legs))):
                bond = legs[i]
                s0, s1 = (int(x) for x in net.bond_site[bond])
                other = s1 if s0 == v else s0
                d = int(net.bond_dim[bond])
                t = np.tensordot(t, m[b, slot[(other, bond)], :d], axes=([i], [0]))
            lz += math.log(abs(float(t)))
        for bond in range(net.n_bonds):
            s0, s1 = (int(x) for x in net.bond_site[bond])
            d = int(net.bond_dim[bond])
            lz -= math.log(abs(float(np.dot(m[b, slot[(s0, bond)], :d], m[b, slot[(s1, bond)], :d]))))
        out.append(lz)
    return out


def test_noalloc_bp_twice_matches_regular_path():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2512_10910_gb300 import build, pne
    from oracle import bp as OB
    build.build()
    ctx = pne.Context(0)
    try:
        cases = [(I.square_lattice(6, 5, 3), [3]), (I.square_lattice(5, 4, 4), [7, 8, 9])]
        for call, (g, seeds) in enumerate(cases):   # two calls in a row
            nets = [I.random_tensors(g, sd) for sd in seeds]
            B = len(nets)
            flat = np.concatenate([n.flat_data()[0] for n in nets])
            data = torch.from_numpy(flat).cuda()
            L = int(g.site_ptr[-1])
            msg = torch.full((B * L * 8,), float("nan"), dtype=torch.float64, device="cuda")
            ns, keep = pne.network_struct(g, data=data, n_batch=B)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            iters, res = pne.pne_bp_messages_noalloc(ns, msg.data_ptr(), 1e-13, 10000)
            torch.cuda.synchronize()
            if call == 1:                            # the call allocated nothing on the device
                assert torch.cuda.mem_get_info()[0] == free0
            assert np.all(iters > 0) and np.all(res < 1e-13)
            host = msg.cpu().numpy()
            g._sets = [n.tensors for n in nets]
            lz = _ln_zbp_from_messages(g, host, B)
            regular = ctx.expand(g, 0, pne.PNE_MODE_LOOP, pne.PNE_F64, data=data, n_batch=B)
            for b in range(B):
                assert abs(lz[b] - regular[b]["log_abs"]) <= 1e-10, (lz[b], regular[b]["log_abs"])
                ref = OB.bp_fixed_point(nets[b])
                for k in range(L):
                    d = len(ref.out[k])
                    np.testing.assert_allclose(host.reshape(B, L, 8)[b, k, :d], ref.out[k], atol=1e-10)
                    assert np.all(host.reshape(B, L, 8)[b, k, d:] == 0.0)
            del keep
    finally:
        ctx.close()


def test_noalloc_rejects_a_network_above_the_scratch_limit():
    # 2 * n_batch * legs * 8 doubles of messages alone exceed the 8 MiB array;
    # the check runs on the host before any CUDA call, so nothing is launched
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2512_10910_gb300 import build, pne
    build.build()
    g = I.square_lattice(4, 4, 2)
    B = 4096
    flat = torch.zeros(B * int(sum(np.prod(g.leg_dims(v)) for v in range(g.n_sites))), dtype=torch.float64,
                       device="cuda")
    ns, keep = pne.network_struct(g, data=flat, n_batch=B)
    msg = torch.empty(B * int(g.site_ptr[-1]) * 8, dtype=torch.float64, device="cuda")
    with pytest.raises(pne.PneError) as e:
        pne.pne_bp_messages_noalloc(ns, msg.data_ptr(), 1e-13, 10000)
    assert e.value.status == pne.PNE_EINVAL and "PNE_NOALLOC_SCRATCH_BYTES" in str(e.value)
    del keep

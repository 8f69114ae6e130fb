"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): every
rank works on its own networks and only the step time crosses ranks -- the
largest over the ranks, by one all-reduce after the timed region -- and each
rank draws different networks (weak scaling, no collective on the data path)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 10.0 + 5.0 * rank                         # this rank's timed total
        got = bench.max_over_ranks(mine, dist, "cpu")
        g, nets = bench.make_networks(bench.WORKLOADS["random16"], rank)
        first = float(nets[0].tensors[0].reshape(-1)[0])
        out.put((rank, got, first, len(nets)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_largest_step_time_and_draw_their_own_networks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][3] == res[1][3] == 32
    assert res[0][2] != res[1][2]                        # rank r takes seeds 32 r .. 32 r + 31
    del torch

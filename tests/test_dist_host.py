"""The multi-GPU bench path is independent replicas: the only cross-rank step
is the max of the ranks' timed regions. Checked here with two gloo ranks on CPU."""

import multiprocessing as mpr
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    got = bench._max_over_ranks(dist, 10.0 + 5.0 * rank, "cpu")
    bench._barrier.__code__  # the barrier helper exists for the timed region
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


def test_max_over_two_gloo_ranks():
    ctx = mpr.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    res = dict(q.get(timeout=5) for _ in range(2))
    assert res == {0: 15.0, 1: 15.0}

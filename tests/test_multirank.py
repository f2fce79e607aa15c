"""Host logic of the N-GPU bench path (replicas, no data-path collective) with
two gloo ranks on the CPU: disjoint road stretches per rank and max-over-ranks
timing."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(10.0 + rank, world, dist, device="cpu")
        q.put((rank, slowest, bench.rank_timesteps(rank, bench.T_COUNT)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_disjoint_stretches_and_the_max_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [11.0, 11.0]          # both ranks report the slowest
    t0, t1 = set(out[0][2]), set(out[1][2])
    assert len(t0) == len(t1) and not (t0 & t1)          # weak scaling: own stretch each


def test_one_rank_is_its_own_maximum():
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5

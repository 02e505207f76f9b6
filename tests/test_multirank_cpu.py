"""The multi-GPU path of bench.py on CPU: world size 2 over gloo.

Products shard across ranks with no data exchange; the only collective is
the max over ranks of the measured duration, and every rank seeds its own
operands."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local = [12.5, 30.0, 7.0, 19.0][rank]
        got = bench.combine_ranks(local, dist)
        seeds = [bench.rank_seed(rank, k) for k in range(4)]
        q.put((rank, got, seeds))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_disjoint_seeds(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = max([12.5, 30.0, 7.0, 19.0][:world])
    assert all(r[1] == want for r in res)
    all_seeds = [s for r in res for s in r[2]]
    assert len(set(all_seeds)) == len(all_seeds)


def test_single_rank_is_identity():
    import bench
    assert bench.combine_ranks(3.25, None) == 3.25

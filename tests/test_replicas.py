"""Multi-process host logic of the replicated (weak-scaling) benchmark, on
CPU with the gloo backend: disjoint episode shards and the timing
reductions."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    os.environ["LOCAL_RANK"] = str(rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1810_00204_gb300 import replicas
    r, lr, ws = replicas.world()
    eps = list(replicas.episode_range(r, ws, 5))
    mx = replicas.reduce_max(10.0 * (rank + 1))
    sm = replicas.reduce_sum(1.5)
    replicas.barrier()
    q.put((rank, lr, ws, eps, mx, sm))
    dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (r0, lr0, ws0, e0, m0, s0), (r1, lr1, ws1, e1, m1, s1) = out
    assert (ws0, ws1) == (2, 2) and (lr0, lr1) == (0, 1)
    assert e0 == [0, 1, 2, 3, 4] and e1 == [5, 6, 7, 8, 9]
    assert m0 == m1 == 20.0
    assert s0 == s1 == 3.0


def test_single_process_is_identity():
    from paper_1810_00204_gb300 import replicas
    assert replicas.reduce_max(3.5) == 3.5
    assert replicas.reduce_sum(2.0) == 2.0
    assert list(replicas.episode_range(0, 1, 3)) == [0, 1, 2]
    with pytest.raises(ValueError):
        replicas.episode_range(2, 2, 3)

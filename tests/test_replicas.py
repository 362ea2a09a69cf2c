"""Multi-rank host logic on CPU (gloo, world size 2): ranks split events with
no data exchange, and only the timing is reduced (max time, summed hits)."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2001_09761_gb300 import gen, replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = gen.batch_sizes(64, 1e3, 1e5, seed=0)
        mine = replicas.strong_split(sizes, world, rank)
        ms, hits = replicas.reduce_timing(10.0 + rank, int(sizes[mine].sum()), dist)
        ws, es = replicas.weak_seeds(rank)
        out.put((rank, sorted(mine.tolist()), ms, hits, ws, es))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes = gen.batch_sizes(64, 1e3, 1e5, seed=0)
    a, b = res[0][1], res[1][1]
    assert not set(a) & set(b) and sorted(a + b) == list(range(64))
    assert res[0][2] == res[1][2] == 11.0             # max over ranks
    assert res[0][3] == res[1][3] == int(sizes.sum())  # summed hits
    la, lb = sizes[a].sum(), sizes[b].sum()
    assert abs(la - lb) <= sizes.max()
    assert res[0][4:] == (0, 1000) and res[1][4:] != res[0][4:]


def test_single_process_reduce_is_identity():
    assert replicas.reduce_timing(3.5, 42, None) == (3.5, 42)
    idx = replicas.strong_split([5, 1, 9], 1, 0)
    assert idx.tolist() == [0, 1, 2]

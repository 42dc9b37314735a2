"""The shard-by-centre decomposition, on CPU ranks with the gloo backend
(world size 2): each rank counts its centres with the oracle's per-centre
Algorithm 1 / Algorithm 2, the cells are all-reduced, and the sum equals the
whole-graph count."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2204_09236_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s, d, t = synth.large(scale=0.0005)
    G = oracle.Graph(s, d, t)
    deg = np.bincount(np.concatenate([s, d]), minlength=G.n)
    cells = np.zeros(56, np.uint64)
    for u in shard.centre_shard(deg, world, rank):
        S, P, Q = G.count_centre(86400, int(u))
        cells += np.concatenate([S.ravel(), P.ravel(), Q.ravel()])
    total = shard.all_reduce_cells(cells, dist)
    if rank == 0:
        q.put(total)
    dist.barrier()
    dist.destroy_process_group()


def test_centre_shards_sum_to_whole_graph():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    total = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    s, d, t = synth.large(scale=0.0005)
    S, P, Q = oracle.count(s, d, t, 86400)
    assert (total == np.concatenate([S.ravel(), P.ravel(), Q.ravel()])).all()
    # Tri types I/III from the summed type II, by the library's host fill
    part = total.copy()
    part[32:40] = 0
    part[48:56] = 0
    filled = shard.fill_tri_types(part)
    assert (filled[32:].reshape(3, 2, 2, 2) == Q).all()
    assert (filled[:32] == total[:32]).all()


def test_shards_partition_the_centres():
    deg = np.random.default_rng(0).integers(0, 50, size=1001)
    parts = [shard.centre_shard(deg, 3, r) for r in range(3)]
    allc = np.sort(np.concatenate(parts))
    assert (allc == np.arange(1001)).all()
    assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1

"""Sharding of the counting work over ranks (multi-GPU design, host side).

Centres are independent (Sec. IV-C, inter-node parallelism): the Star/Pair
counters and the Tri type-II counters of a graph are sums over centres. A
rank that counts the centres of its shard (tm_count_centres) and an
all-reduce of the 56 cells therefore give the whole graph's counters; the Tri
type-I/III cells are filled from the summed type-II cells afterwards, by the
library.

This module only assigns centres and sums cells; it runs no counting.
"""
from __future__ import annotations

import numpy as np


def centre_shard(degrees, world, rank):
    """Centres of `rank`: the centres sorted by degree are dealt round-robin,
    so every rank gets a similar mix of hubs and leaves."""
    order = np.argsort(-np.asarray(degrees), kind="stable")
    return np.sort(order[rank::world])


def all_reduce_cells(cells, dist=None):
    """Sum of a uint64[56] cell vector over the ranks (torch.distributed with
    any backend; None for a single rank)."""
    cells = np.asarray(cells, np.uint64)
    if dist is None:
        return cells
    import torch
    t = torch.from_numpy(cells.astype(np.int64))  # sums stay below 2^63 here
    if dist.get_backend() == "nccl":
        t = t.cuda()  # NCCL reduces device tensors
    dist.all_reduce(t)
    return t.cpu().numpy().astype(np.uint64)


def fill_tri_types(cells):
    """The summed 56 cells with the Tri type-I/III cells filled from type II,
    by the library (tm_fill_tri_types)."""
    from . import tm
    return tm.fill_tri_types(cells)

"""Splitting interface nodes across ranks.

Interface values are independent of one another (Sec. 5 of the paper), so the
nodes of a request shard across processes with no exchange on the data path:
each rank evaluates a contiguous range of nodes under their global node ids
(so every walk keeps its Philox stream) and the per-node results are gathered
afterwards.  One process per GPU; nothing here launches GPU work.
"""
from __future__ import annotations

import numpy as np


def shard_range(n_nodes: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous node range [begin, end) of `rank`; sizes differ by at most one."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    base, extra = divmod(n_nodes, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def shard(nodes, n_paths, rank: int, world: int):
    """The rank's nodes, path counts and global node ids."""
    nodes = np.asarray(nodes, dtype=np.float64).reshape(-1, 2)
    npth = np.asarray(n_paths, dtype=np.int64)
    if npth.ndim == 0:
        npth = np.full(len(nodes), int(npth), dtype=np.int64)
    b, e = shard_range(len(nodes), rank, world)
    return nodes[b:e], npth[b:e], np.arange(b, e, dtype=np.uint32)


def gather(local: np.ndarray, n_nodes: int, rank: int, world: int, dist):
    """All-gather per-node arrays [n_local, ...] into [n_nodes, ...] in node
    order (torch.distributed, any backend that all_gathers CPU tensors)."""
    import torch
    b, e = shard_range(n_nodes, rank, world)
    tail = local.shape[1:]
    width = max(shard_range(n_nodes, r, world)[1] - shard_range(n_nodes, r, world)[0]
                for r in range(world))
    buf = np.zeros((width,) + tail, dtype=local.dtype)
    buf[: e - b] = local
    t = torch.from_numpy(buf)
    parts = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    out = np.zeros((n_nodes,) + tail, dtype=local.dtype)
    for r in range(world):
        rb, re_ = shard_range(n_nodes, r, world)
        out[rb:re_] = parts[r].numpy()[: re_ - rb]
    return out

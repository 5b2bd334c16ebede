"""One evaluation split across ranks by (node, path-range) units.

Interface values are independent of one another, and so are the walks of
one node (Sec. 5), so an evaluation shards at any granularity.  The unit
here is a range: a node and a contiguous range of its paths.

1. Every rank builds the same list of ranges (`ranges`): node by node, each
   node's paths in order, at most `chunk` paths per range.
2. It takes a contiguous slice of that list (`balance`), the slices cut so
   that their expected Euler steps are about equal.  A range costs its
   paths x the node's mean exit time (`mean_exit_time`).
3. It evaluates its slice with sdd_range_sums / sdd_range_sums_device (raw
   FP64 sums per range) into its rows of a table [n_ranges][E][4] whose
   other rows are zero, and likewise for the walk counts.
4. One all-reduce SUM per table (`allreduce_table`) hands every rank the
   whole table exactly: each row has one nonzero contribution, and
   x + 0 = x in floating point.
5. sdd_reduce_sums adds each node's ranges in range order and forms the
   mean and standard errors.

Given the range list, the result does not depend on the number of ranks or
on their slices.  One process per GPU; nothing here launches GPU work.
"""
from __future__ import annotations

import numpy as np


def ranges(n_paths, chunk: int):
    """The range list of an evaluation with n_paths[j] walks at node j:
    (node [m], begin [m], count [m]) int64 arrays, node by node, at most
    `chunk` paths per range, each node's ranges in path order."""
    npth = np.asarray(n_paths, dtype=np.int64).ravel()
    if chunk < 1:
        raise ValueError("chunk must be >= 1")
    per = (npth + chunk - 1) // chunk
    node = np.repeat(np.arange(len(npth), dtype=np.int64), per)
    first = np.concatenate([[0], np.cumsum(per)[:-1]]) if len(per) else np.zeros(0, np.int64)
    k = np.arange(len(node), dtype=np.int64) - np.repeat(first, per)
    begin = k * chunk
    count = np.minimum(chunk, npth[node] - begin)
    return node, begin, count


def mean_exit_time(nodes, domain, terms: int = 61):
    """E[tau] of a standard 2D Brownian motion started at each node, stopped
    at the rectangle's boundary: the separation-of-variables series of
    (1/2) Lap T = -1, T = 0 on the boundary, over odd modes up to `terms`.
    Used only to balance work (a TE walk is that Brownian motion)."""
    xmin, xmax, zmin, zmax = domain
    W, H = xmax - xmin, zmax - zmin
    p = np.asarray(nodes, dtype=np.float64).reshape(-1, 2)
    m = np.arange(1, terms + 1, 2, dtype=np.float64)
    M, N = np.meshgrid(m, m, indexing="ij")
    lam = 0.5 * np.pi ** 2 * ((M / W) ** 2 + (N / H) ** 2)
    coef = 16.0 / (np.pi ** 2 * M * N * lam)
    sx = np.sin(np.pi * np.outer(p[:, 0] - xmin, m) / W)  # [n][modes]
    sz = np.sin(np.pi * np.outer(p[:, 1] - zmin, m) / H)
    return np.maximum(np.einsum("im,mn,in->i", sx, coef, sz), 0.0)


def balance(cost, world: int):
    """Boundaries b[0] = 0 <= ... <= b[world] = len(cost) of contiguous
    slices: rank r takes ranges b[r] .. b[r+1]-1, the cut put where the
    cumulative cost crosses r / world of the total."""
    c = np.asarray(cost, dtype=np.float64).ravel()
    if world < 1:
        raise ValueError("world must be >= 1")
    if len(c) == 0:
        return np.zeros(world + 1, dtype=np.int64)
    cum = np.cumsum(c)
    total = cum[-1]
    b = [0]
    for r in range(1, world):
        # first range whose cumulative cost reaches r / world of the total
        b.append(int(np.searchsorted(cum, total * r / world, side="left")))
    b.append(len(c))
    return np.maximum.accumulate(np.asarray(b, dtype=np.int64))


def plan(nodes, n_paths, chunk: int, world: int, domain):
    """Ranges of an evaluation and the slice boundaries of `world` ranks."""
    node, begin, count = ranges(n_paths, chunk)
    tau = mean_exit_time(nodes, domain)
    bounds = balance(count * np.maximum(tau[node], 1e-12), world)
    return {"node": node, "begin": begin, "count": count, "bounds": bounds}


def allreduce_table(table, dist):
    """SUM all-reduce of a table in which every row has exactly one rank's
    nonzero contribution (torch tensor, in place): the result is exact."""
    dist.all_reduce(table, op=dist.ReduceOp.SUM)
    return table

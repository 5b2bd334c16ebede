"""One evaluation split across ranks (gloo, world sizes 2 and 3, CPU).

Each rank evaluates its cost-balanced slice of the (node, path-range) list
with the oracle's range sums, writes them into its rows of a zero table, and
one all-reduce SUM gives every rank the whole table.  The table must equal
the single-process table bit for bit, and so must the node means formed
from it in range order.
"""
import os
import socket

import numpy as np
import pytest

from paper_1603_09311_gb300 import inputs as I
from paper_1603_09311_gb300 import shard as S

CHUNK = 256


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _job():
    w = I.scaled(I.workload("quarterspace"), n_nodes=7, paths_per_node=1500, dt=1e-3)
    w["n_paths"] = np.array([1500, 700, 1, 256, 257, 1100, 900], dtype=np.int64)  # ragged
    return w


def _node_means(node, sums, nvalid, n_nodes):
    # fixed-order per-node reduction (range order) of a table
    mean = np.full((n_nodes,) + sums.shape[1:2], np.nan + 0j)
    for j in range(n_nodes):
        rows = np.flatnonzero(node == j)
        acc = np.zeros(sums.shape[1:])
        nv = 0
        for r in rows:
            acc = acc + sums[r]
            nv += int(nvalid[r])
        mean[j] = (acc[:, 0] + 1j * acc[:, 1]) / nv
    return mean


def _worker(rank, world, port, out_dir):
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from oracle import oracle as O
    from paper_1603_09311_gb300 import shard as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _job()
    P = S.plan(w["nodes"], w["n_paths"], CHUNK, world, I.DOMAIN)
    b, e = int(P["bounds"][rank]), int(P["bounds"][rank + 1])
    n = len(P["node"])
    table = torch.zeros((n, 1, 4), dtype=torch.float64)
    nvalid = torch.zeros(n, dtype=torch.int64)
    if e > b:
        sl = slice(b, e)
        sums, nv, _ = O.range_sums(w["model"], w["nodes"][P["node"][sl]], P["node"][sl], P["begin"][sl],
                                   P["count"][sl], w["dt"], w["seed"], threads=2)
        table[b:e] = torch.from_numpy(sums)
        nvalid[b:e] = torch.from_numpy(nv)
    S.allreduce_table(table, dist)
    S.allreduce_table(nvalid, dist)
    np.save(os.path.join(out_dir, f"table{rank}.npy"), table.numpy())
    np.save(os.path.join(out_dir, f"nvalid{rank}.npy"), nvalid.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_ranges_cover_every_path_once():
    for npth, chunk in (([1500, 1, 256, 257, 0, 3], 256), ([5, 5], 1), ([], 8), ([10 ** 6], 4096)):
        node, begin, count = S.ranges(npth, chunk)
        assert np.all(count >= 1) and np.all(count <= chunk)
        for j, n in enumerate(npth):
            rows = np.flatnonzero(node == j)
            assert np.all(np.diff(rows) == 1)  # a node's ranges are contiguous ...
            got = np.concatenate([np.arange(b, b + c) for b, c in zip(begin[rows], count[rows])]) if len(rows) else []
            assert np.array_equal(got, np.arange(n))  # ... and cover its paths in order
        assert np.all(np.diff(node) >= 0)


def test_balance_cuts_contiguous_slices_of_equal_cost():
    rng = np.random.default_rng(0)
    cost = rng.exponential(1.0, 1000)
    for world in (1, 2, 3, 8):
        b = S.balance(cost, world)
        assert b[0] == 0 and b[-1] == len(cost) and np.all(np.diff(b) >= 0)
        share = np.array([cost[b[r]:b[r + 1]].sum() for r in range(world)])
        # each slice is within one range's cost of its fair share
        assert np.all(np.abs(share - cost.sum() / world) <= cost.max() + 1e-9), share
    assert np.array_equal(S.balance([], 4), np.zeros(5, dtype=np.int64))


def test_mean_exit_time_of_the_cost_model():
    # the series solves (1/2) Lap T = -1 with T = 0 on the walls: check the
    # equation by finite differences and the boundary values
    dom = I.DOMAIN
    h = 1e-3
    for x, z in ((0.0, 0.25), (0.5, 0.6), (-0.8, -0.3)):
        pts = [(x, z), (x + h, z), (x - h, z), (x, z + h), (x, z - h)]
        T = S.mean_exit_time(pts, dom, terms=401)
        lap = (T[1] + T[2] + T[3] + T[4] - 4 * T[0]) / h ** 2
        assert abs(0.5 * lap + 1.0) < 2e-2, lap
    edge = S.mean_exit_time([(-1.0, 0.3), (1.0, 0.3), (0.2, -0.5), (0.2, 1.0)], dom)
    assert np.all(np.abs(edge) < 1e-9)


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_reproduce_one_process(tmp_path, world):
    # the table, and the node means formed from it, do not depend on the
    # number of ranks or on their slices
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from oracle import oracle as O
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True, start_method="spawn")
    w = _job()
    P = S.plan(w["nodes"], w["n_paths"], CHUNK, world, I.DOMAIN)
    # every rank holds a nonempty slice
    assert np.all(np.diff(P["bounds"]) > 0)
    sums, nv, _ = O.range_sums(w["model"], w["nodes"][P["node"]], P["node"], P["begin"], P["count"],
                               w["dt"], w["seed"], threads=3)
    for r in range(world):
        t = np.load(tmp_path / f"table{r}.npy")
        n = np.load(tmp_path / f"nvalid{r}.npy")
        assert np.array_equal(t, sums) and np.array_equal(n, nv)
    # node means from the table, in range order, equal the one-process ones
    # and agree with the oracle's whole-node evaluation (other summation order)
    mean = _node_means(P["node"], np.load(tmp_path / "table1.npy"), np.load(tmp_path / "nvalid1.npy"), 7)
    assert np.array_equal(mean, _node_means(P["node"], sums, nv, 7))
    ref = O.interface_values(w["model"], w["nodes"], w["n_paths"], w["dt"], w["seed"], threads=2)
    assert np.allclose(mean, ref["mean"], rtol=1e-13, atol=1e-15)

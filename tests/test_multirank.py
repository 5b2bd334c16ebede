"""Sharding across ranks (gloo, world size 2, CPU): each rank evaluates its
contiguous share of the nodes under their global node ids with the oracle,
and the gathered result equals the single-process evaluation exactly."""
import os
import socket

import numpy as np
import pytest

from paper_1603_09311_gb300 import shard as S


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from oracle import oracle as O
    from paper_1603_09311_gb300 import inputs as I
    from paper_1603_09311_gb300 import shard as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = I.scaled(I.workload("quarterspace"), n_nodes=7, paths_per_node=1500, dt=1e-3)
    nodes, npth, ids = S.shard(w["nodes"], w["n_paths"], rank, world)
    r = O.interface_values(w["model"], nodes, npth, w["dt"], w["seed"], node_id0=int(ids[0]), threads=2)
    mean = np.stack([r["mean"].real, r["mean"].imag], -1)
    full_mean = S.gather(mean, len(w["nodes"]), rank, world, dist)
    full_se = S.gather(r["se"], len(w["nodes"]), rank, world, dist)
    if rank == 0:
        np.save(os.path.join(out_dir, "mean.npy"), full_mean)
        np.save(os.path.join(out_dir, "se.npy"), full_se)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_cover_every_node_once():
    for n in (0, 1, 5, 64, 257):
        for world in (1, 2, 3, 8):
            got = []
            for r in range(world):
                b, e = S.shard_range(n, r, world)
                got.extend(range(b, e))
                assert e - b in (n // world, n // world + 1)
            assert got == list(range(n))


def test_two_ranks_reproduce_one_process(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from oracle import oracle as O
    from paper_1603_09311_gb300 import inputs as I
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    w = I.scaled(I.workload("quarterspace"), n_nodes=7, paths_per_node=1500, dt=1e-3)
    ref = O.interface_values(w["model"], w["nodes"], w["n_paths"], w["dt"], w["seed"], threads=2)
    mean = np.load(tmp_path / "mean.npy")
    se = np.load(tmp_path / "se.npy")
    assert np.array_equal(mean[..., 0] + 1j * mean[..., 1], ref["mean"])
    assert np.array_equal(se, ref["se"])

"""Work items of one evaluation (host logic, no GPU).

The node values are independent (Sec. 5), so an evaluation is cut into
(node, path range) items that the persistent warps take from one queue.  The
walks and their sums are only right if every path of every node is in
exactly one item; the queue only drains evenly if the guided items shrink
toward its end, also when the nodes outnumber the warps.
"""
import numpy as np
import pytest

from paper_1603_09311_gb300 import build as B
from paper_1603_09311_gb300 import sdd


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    sdd.lib()


def _cmin(n_paths):
    # the smallest guided item: 32 paths, or total / 2^20 rounded up to 32
    return max(32, (int(np.sum(n_paths)) // (1 << 20) + 31) // 32 * 32)


def _check_cover(n_paths, node, path0, count):
    assert np.all(count > 0)
    for j, n in enumerate(n_paths):
        sel = node == j
        p, c = path0[sel].astype(np.int64), count[sel].astype(np.int64)
        o = np.argsort(p)
        p, c = p[o], c[o]
        if n == 0:
            assert len(p) == 0
            continue
        # contiguous, no gap and no overlap, from 0 to n
        assert p[0] == 0 and np.all(p[1:] == p[:-1] + c[:-1]) and p[-1] + c[-1] == n


def _final_piece(n_paths, node, path0, count):
    return path0.astype(np.int64) + count == np.asarray(n_paths, dtype=np.int64)[node]


@pytest.mark.parametrize("n_paths,warps,factor", [
    (np.full(64, 100_000), 152 * 32, 4),            # the quarter-space line on 152 SMs
    (np.full(16, 10_000), 456 * 8, 2),
    (np.array([1, 31, 33, 700, 2049, 0, 5]), 64, 2),  # ragged and empty nodes
    (np.full(3000, 20_000), 456 * 8, 2),            # more nodes than the warps can share
    (np.exp(np.random.default_rng(3).uniform(np.log(1e4), np.log(1e6), 256)).astype(np.int64), 1216 * 4, 8),
])
def test_guided_items_cover_every_path_once_and_shrink(n_paths, warps, factor):
    node, path0, count = sdd.sdd_plan_items(n_paths, warps, factor)
    _check_cover(n_paths, node, path0, count)
    fin = _final_piece(n_paths, node, path0, count)
    # every item but a node's last piece is a multiple of 32 paths
    assert np.all(count[~fin] % 32 == 0)
    # sizes never grow along the queue (a node's last piece may be smaller)
    full = count[~fin]
    assert np.all(full[1:] <= full[:-1])
    # the end of the queue is down to the smallest item
    assert count[-1] <= _cmin(n_paths)
    if len(count) > 2 * warps:
        assert count[:warps].max() >= 4 * count[-warps:].max()


def test_fixed_chunks_node_by_node():
    n_paths = np.array([100, 0, 64, 65])
    node, path0, count = sdd.sdd_plan_items(n_paths, 8, 1, chunk_paths=32)
    _check_cover(n_paths, node, path0, count)
    assert list(node) == [0, 0, 0, 0, 2, 2, 3, 3, 3]
    assert list(count) == [32, 32, 32, 4, 32, 32, 32, 32, 1]


def test_no_nodes_and_bad_arguments():
    node, path0, count = sdd.sdd_plan_items(np.zeros(0, dtype=np.int64), 8)
    assert len(node) == 0
    for kw in ({"warps": 0}, {"warps": 8, "guided_factor": 0}, {"warps": 8, "chunk_paths": -1}):
        with pytest.raises(sdd.SddError) as e:
            sdd.sdd_plan_items(np.full(2, 10), **kw)
        assert e.value.status == sdd.SDD_E_ARG
    with pytest.raises(sdd.SddError):
        sdd.sdd_plan_items(np.array([10, -1]), 8)

"""Range sums and their reduction on the GPU, through the C ABI: the units of
an evaluation split across processes.

- FP64 mode: every range's raw sums equal the oracle's range sums to 1e-10
  of the largest |sum| scale (same streams), walk counts exactly.
- A slice-by-slice evaluation (the ranks of a 3-way split, each its own
  call), combined in a zero-padded table, equals the evaluation of all
  ranges in one call up to the FP64 summation order within a range.
- The reduction equals the whole-node entry point on the same walks.
- Device and host entry points agree; argument errors are reported.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1603_09311_gb300 import build as B
from paper_1603_09311_gb300 import inputs as I
from paper_1603_09311_gb300 import sdd
from paper_1603_09311_gb300 import shard as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    sdd.lib()


def _job(name="quarterspace", n_nodes=8, paths=3000, dt=1e-3):
    w = I.scaled(I.workload(name), n_nodes=n_nodes, paths_per_node=paths, dt=dt)
    w["n_paths"] = w["n_paths"].copy()
    w["n_paths"][::3] += 517  # ragged: partial ranges
    return w


@pytest.mark.parametrize("name", ["quarterspace", "block"])
def test_fp64_range_sums_equal_oracle(name):
    w = _job(name, n_nodes=5, paths=900)
    P = S.plan(w["nodes"], w["n_paths"], 256, 1, I.DOMAIN)
    ctx = sdd.sdd_create(w["model"])
    sums, nv, st = sdd.sdd_range_sums(ctx, w["nodes"][P["node"]], P["begin"], P["count"], w["dt"], w["seed"],
                                      node_ids=P["node"], precision="fp64")
    ref, rnv, rsteps = O.range_sums(w["model"], w["nodes"][P["node"]], P["node"], P["begin"], P["count"],
                                    w["dt"], w["seed"], urule=32)
    assert np.array_equal(nv, rnv) and st["steps"] == rsteps
    scale = np.abs(ref).max(axis=0, keepdims=True)
    assert np.all(np.abs(sums - ref) <= 1e-10 * np.maximum(scale, 1.0))


def test_sliced_evaluation_equals_one_call_and_the_whole_node_call():
    w = _job()
    n = len(w["nodes"])
    ctx = sdd.sdd_create(w["model"])
    P = S.plan(w["nodes"], w["n_paths"], 512, 3, I.DOMAIN)
    node, begin, count, b = P["node"], P["begin"], P["count"], P["bounds"]
    full, fnv, _ = sdd.sdd_range_sums(ctx, w["nodes"][node], begin, count, w["dt"], w["seed"], node_ids=node)
    table = np.zeros_like(full)
    tnv = np.zeros_like(fnv)
    for r in range(3):
        sl = slice(int(b[r]), int(b[r + 1]))
        assert b[r + 1] > b[r]
        s_, v_, _ = sdd.sdd_range_sums(ctx, w["nodes"][node[sl]], begin[sl], count[sl], w["dt"], w["seed"],
                                       node_ids=node[sl])
        part = np.zeros_like(full)
        part[sl] = s_
        table = table + part  # the all-reduce SUM of zero-padded tables
        pv = np.zeros_like(fnv)
        pv[sl] = v_
        tnv = tnv + pv
    assert np.array_equal(tnv, fnv)
    assert np.allclose(table, full, rtol=1e-13, atol=0)
    mean, se = sdd.sdd_reduce_sums(ctx, n, node, table, tnv)
    ref, rse, _ = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], w["dt"], w["seed"])
    scale = np.abs(ref).max()
    assert np.allclose(mean, ref, rtol=0, atol=1e-12 * scale)
    assert np.allclose(se, rse, rtol=1e-9, atol=0)


def test_device_entry_points_match_host_ones():
    torch = pytest.importorskip("torch")
    w = _job(n_nodes=6, paths=2000)
    ctx = sdd.sdd_create(w["model"])
    P = S.plan(w["nodes"], w["n_paths"], 700, 1, I.DOMAIN)
    node, begin, count = P["node"], P["begin"], P["count"]
    m = len(node)
    hs, hv, _ = sdd.sdd_range_sums(ctx, w["nodes"][node], begin, count, w["dt"], 9, node_ids=node)
    hm, hse = sdd.sdd_reduce_sums(ctx, 6, node, hs, hv)
    dev = torch.device("cuda:0")
    d_nodes = torch.tensor(w["nodes"][node], dtype=torch.float64, device=dev)
    d_ids = torch.tensor(node.astype(np.int32), device=dev)
    d_sums = torch.empty((m, ctx.E, 4), dtype=torch.float64, device=dev)
    d_nv = torch.empty(m, dtype=torch.int64, device=dev)
    d_cnt = torch.zeros(3, dtype=torch.int64, device=dev)
    d_mean = torch.empty((6, ctx.E, 2), dtype=torch.float64, device=dev)
    d_se = torch.empty_like(d_mean)
    stream = torch.cuda.current_stream().cuda_stream
    sdd.sdd_range_sums_device(ctx, d_nodes.data_ptr(), m, begin, count, w["dt"], 9, d_sums.data_ptr(),
                              d_nv.data_ptr(), d_node_ids_ptr=d_ids.data_ptr(), d_counters_ptr=d_cnt.data_ptr(),
                              stream=stream)
    sdd.sdd_reduce_sums_device(ctx, 6, node, d_sums.data_ptr(), d_nv.data_ptr(), d_mean.data_ptr(),
                               d_se.data_ptr(), stream=stream)
    torch.cuda.synchronize()
    assert np.array_equal(d_nv.cpu().numpy(), hv) and int(d_cnt[1]) == int(count.sum())
    assert np.allclose(d_sums.cpu().numpy(), hs, rtol=1e-13, atol=0)
    dm = d_mean.cpu().numpy()
    assert np.allclose(dm[..., 0] + 1j * dm[..., 1], hm, rtol=0, atol=1e-12 * np.abs(hm).max())
    assert np.allclose(d_se.cpu().numpy(), hse, rtol=1e-9, atol=0)


def test_range_arguments_and_empty_nodes():
    w = _job(n_nodes=3, paths=100)
    ctx = sdd.sdd_create(w["model"])
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_range_sums(ctx, w["nodes"][:1], [2 ** 32 - 10], [11], w["dt"], 0)
    assert e.value.status == sdd.SDD_E_ARG
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_range_sums(ctx, w["nodes"][:1], [0], [10], w["dt"], 0, use_graph=1)
    assert e.value.status == sdd.SDD_E_UNSUPPORTED
    # a range at the top of the 32-bit path space is fine
    s_, v_, _ = sdd.sdd_range_sums(ctx, w["nodes"][:1], [2 ** 32 - 10], [10], w["dt"], 0)
    assert v_[0] == 10
    sums = np.ones((2, 1, 4))
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_reduce_sums(ctx, 3, [1, 0], sums, [1, 1])  # not nondecreasing
    assert e.value.status == sdd.SDD_E_ARG
    # node 1 without ranges: NaN mean and standard error; node 2 one walk: NaN se
    mean, se = sdd.sdd_reduce_sums(ctx, 3, [0, 0, 2], np.ones((3, 1, 4)), [2, 3, 1])
    assert mean[0, 0] == 2 / 5 + 2j / 5 and np.isnan(mean[1, 0]) and np.all(np.isnan(se[1]))
    assert mean[2, 0] == 1 + 1j and np.all(np.isnan(se[2]))

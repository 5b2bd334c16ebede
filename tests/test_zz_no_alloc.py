"""The entry point for callers that cannot allocate device memory.

sdd_interface_values_noalloc serves callers that must not call cudaMalloc
(hosts that hand out all device memory from their own arena, processes whose
memory another framework's caching allocator already holds, loops that cannot
afford the synchronisation of an allocation).  It runs the same walks as
sdd_interface_values_device with its scratch in a fixed array inside the
library, so on the same inputs it must give the same node values, up to the
order of the FP64 sums.  Two calls in a row with different requests check
that the second is not disturbed by what the first left in the shared array.
This file is collected last so that a stopping run has already run every
other test.
"""
import numpy as np
import pytest

from paper_1603_09311_gb300 import build as B
from paper_1603_09311_gb300 import inputs as I
from paper_1603_09311_gb300 import sdd

pytestmark = pytest.mark.gpu

REL = 1e-12  # same walks; only the summation order of the FP64 sums may differ


def _buffers(torch, w, E):
    dev = torch.device("cuda:0")
    n = len(w["nodes"])
    return {
        "nodes": torch.tensor(w["nodes"], dtype=torch.float64, device=dev),
        "mean": torch.empty((n, E, 2), dtype=torch.float64, device=dev),
        "se": torch.empty((n, E, 2), dtype=torch.float64, device=dev),
        "cnt": torch.zeros(3, dtype=torch.int64, device=dev),
        "mean2": torch.empty((n, E, 2), dtype=torch.float64, device=dev),
        "se2": torch.empty((n, E, 2), dtype=torch.float64, device=dev),
        "cnt2": torch.zeros(3, dtype=torch.int64, device=dev),
    }


def _run(fn, ctx, w, b, mean, se, cnt, stream):
    fn(ctx, b["nodes"].data_ptr(), len(w["nodes"]), w["n_paths"], w["dt"], w["seed"],
       b[mean].data_ptr(), b[se].data_ptr(), d_counters_ptr=b[cnt].data_ptr(),
       stream=stream.cuda_stream, **w.get("cfg", {}))


def test_no_alloc_entry_point_matches_the_allocating_one():
    torch = pytest.importorskip("torch")
    B.build()
    sdd.lib()
    stream = torch.cuda.current_stream()
    first = I.scaled(I.workload("quarterspace"), n_nodes=64, paths_per_node=3000, dt=1e-3)
    first["seed"] = 11
    second = I.scaled(I.workload("block"), n_nodes=40, paths_per_node=2000, dt=1e-3)
    second["seed"] = 12
    # 64 nodes x 5003 walks in chunks of 32 would need 10048 work items, more
    # than SDD_NOALLOC_MAX_ITEMS: the call widens its chunks to 40 walks (8064
    # items, the last of each node 3 walks)
    third = I.scaled(I.workload("quarterspace"), n_nodes=64, paths_per_node=5003, dt=1e-3)
    third["seed"] = 13
    third["cfg"] = {"chunk_paths": 32}
    cases = []
    for w in (first, second, third):
        ctx = sdd.sdd_create(w["model"])
        b = _buffers(torch, w, ctx.E)
        # reference: the allocating device entry point
        _run(sdd.sdd_interface_values_device, ctx, w, b, "mean", "se", "cnt", stream)
        torch.cuda.synchronize()
        cases.append((ctx, w, b))

    free_before = None
    for k, (ctx, w, b) in enumerate(cases):
        if k == 1:
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
        _run(sdd.sdd_interface_values_noalloc, ctx, w, b, "mean2", "se2", "cnt2", stream)
        torch.cuda.synchronize()
        ref_m, got_m = b["mean"].cpu().numpy(), b["mean2"].cpu().numpy()
        ref_s, got_s = b["se"].cpu().numpy(), b["se2"].cpu().numpy()
        scale = np.abs(ref_m).max()
        assert np.allclose(got_m, ref_m, rtol=0, atol=REL * scale), f"call {k + 1}: means differ"
        assert np.allclose(got_s, ref_s, rtol=1e-9, atol=0), f"call {k + 1}: standard errors differ"
        assert np.array_equal(b["cnt2"].cpu().numpy(), b["cnt"].cpu().numpy()), f"call {k + 1}"
    # the second call allocated nothing on the device
    assert torch.cuda.mem_get_info()[0] == free_before

    # more nodes than the fixed scratch holds: a clear argument error, no work
    ctx, w, b = cases[0]
    with pytest.raises(sdd.SddError) as err:
        sdd.sdd_interface_values_noalloc(ctx, b["nodes"].data_ptr(), len(w["nodes"]), w["n_paths"], w["dt"], 1,
                                         b["mean2"].data_ptr(), b["se2"].data_ptr(), use_graph=1)
    assert err.value.status == sdd.SDD_E_UNSUPPORTED
    many = sdd.lib().sdd_interface_values_noalloc
    n_big = 4097
    npth = np.ones(n_big, dtype=np.int64)
    st = many(ctx.handle, b["nodes"].data_ptr(), None, n_big,
              npth.ctypes.data_as(sdd.P(sdd.ctypes.c_int64)), 1e-3, 0, None,
              b["mean2"].data_ptr(), b["se2"].data_ptr(), None, None)
    assert st == sdd.SDD_E_ARG
    assert "SDD_NOALLOC_MAX_NODES" in sdd.sdd_last_error()
    for c, _, _ in cases:
        c.close()

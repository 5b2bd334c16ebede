"""Asynchronous requests through the C ABI (sdd_interface_values_async,
sdd_poll, sdd_wait, sdd_cancel, sdd_request_result, sdd_request_free).

A request runs the walks of sdd_interface_values on the same plan, so its
result equals the synchronous call's up to the FP64 summation order within a
work item.  Several requests of one context may be in flight on several
streams and be submitted from several host threads; a cancelled request
ends early with SDD_E_CANCELLED.
"""
import threading
import time

import numpy as np
import pytest

from paper_1603_09311_gb300 import build as B
from paper_1603_09311_gb300 import inputs as I
from paper_1603_09311_gb300 import sdd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    sdd.lib()


def _close(a, b):
    scale = max(1.0, np.abs(b).max())
    return np.allclose(a, b, rtol=0, atol=1e-12 * scale)


def test_async_result_equals_the_synchronous_call():
    w = I.scaled(I.workload("block"), n_nodes=12, paths_per_node=4000, dt=1e-3)
    ctx = sdd.sdd_create(w["model"])
    ref, rse, rst = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], w["dt"], 5)
    req = sdd.sdd_interface_values_async(ctx, w["nodes"], w["n_paths"], w["dt"], 5)
    assert req.wait() == sdd.SDD_OK
    m, se, st = req.result()
    assert _close(m, ref) and np.allclose(se, rse, rtol=1e-9, atol=0)
    assert st["walks"] == rst["walks"] and st["steps"] == rst["steps"]
    req.free()
    # an empty request ends at once
    e = sdd.sdd_interface_values_async(ctx, np.zeros((0, 2)), np.zeros(0, dtype=np.int64), 1e-3, 0)
    assert e.wait() == sdd.SDD_OK and e.result()[0].shape == (0, 16)


def test_requests_in_flight_together_on_several_streams():
    torch = pytest.importorskip("torch")
    w = I.scaled(I.workload("quarterspace"), n_nodes=16, paths_per_node=20000, dt=1e-3)
    ctx = sdd.sdd_create(w["model"])
    streams = [torch.cuda.Stream() for _ in range(3)]
    seeds = [11, 12, 13, 14]
    reqs = [sdd.sdd_interface_values_async(ctx, w["nodes"], w["n_paths"], w["dt"], sd,
                                           stream=(streams[k].cuda_stream if k < 3 else 0))
            for k, sd in enumerate(seeds)]
    for sd, r in zip(seeds, reqs):
        assert r.wait() == sdd.SDD_OK
        m, se, _ = r.result()
        ref, rse, _ = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], w["dt"], sd)
        assert _close(m, ref) and np.allclose(se, rse, rtol=1e-9, atol=0)
        r.free()


def test_submission_from_several_threads():
    w = I.scaled(I.workload("triangle"), n_nodes=8, paths_per_node=10000, dt=1e-3)
    ctx = sdd.sdd_create(w["model"])
    out, errors = {}, []

    def worker(k):
        try:
            reqs = [sdd.sdd_interface_values_async(ctx, w["nodes"], w["n_paths"], w["dt"], 100 * k + j)
                    for j in range(3)]
            for j, r in enumerate(reqs):
                assert r.wait() == sdd.SDD_OK
                out[(k, j)] = r.result()[0]
                r.free()
        except Exception as exc:  # reported below
            errors.append(exc)

    th = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    for (k, j), m in out.items():
        ref, _, _ = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], w["dt"], 100 * k + j)
        assert _close(m, ref)


def test_poll_timeout_and_cancel():
    # a request of about a second (64 nodes x 2e6 walks at dt 1e-4 would be
    # longer; the quarter-space line at 2e5 walks per node takes ~0.1 s per
    # 1e5): poll reports it running, a short wait times out, and a cancel
    # after it has started ends it well before its full time
    w = I.workload("quarterspace")
    npth = np.full(64, 2_000_000, dtype=np.int64)
    ctx = sdd.sdd_create(w["model"])
    t0 = time.perf_counter()
    req = sdd.sdd_interface_values_async(ctx, w["nodes"], npth, w["dt"], 3)
    assert req.poll() == sdd.SDD_E_BUSY
    assert req.wait(50) == sdd.SDD_E_TIMEOUT
    assert req.cancel() == sdd.SDD_OK
    assert req.wait() == sdd.SDD_E_CANCELLED
    t_cancel = time.perf_counter() - t0
    with pytest.raises(sdd.SddError) as e:
        req.result()
    assert e.value.status == sdd.SDD_E_CANCELLED
    assert req.cancel() == sdd.SDD_OK  # a second cancel is harmless
    req.free()
    # the same request left to run takes far longer
    t0 = time.perf_counter()
    full = sdd.sdd_interface_values_async(ctx, w["nodes"], npth, w["dt"], 3)
    assert full.wait() == sdd.SDD_OK
    t_full = time.perf_counter() - t0
    _, _, st = full.result()
    assert st["walks"] == npth.sum()
    full.free()
    assert t_cancel < 0.5 * t_full, (t_cancel, t_full)


def test_a_cancel_made_while_queued_behind_another_request_is_kept():
    # request b waits on the stream behind a (64 nodes x 2e6 walks, about a
    # second); b is cancelled before its queue memset has run, then a.  The
    # cancel of b must survive that memset: b's warps take at most one walk
    # per lane before the flag arrives, so b ends right after a instead of
    # running its own second of walks
    torch = pytest.importorskip("torch")
    w = I.workload("quarterspace")
    npth = np.full(64, 2_000_000, dtype=np.int64)
    ctx = sdd.sdd_create(w["model"])
    s = torch.cuda.Stream()
    a = sdd.sdd_interface_values_async(ctx, w["nodes"], npth, w["dt"], 3, stream=s.cuda_stream)
    b = sdd.sdd_interface_values_async(ctx, w["nodes"], npth, w["dt"], 4, stream=s.cuda_stream)
    assert b.cancel() == sdd.SDD_OK
    time.sleep(0.05)
    assert a.cancel() == sdd.SDD_OK
    assert a.wait() == sdd.SDD_E_CANCELLED
    t0 = time.perf_counter()
    assert b.wait() == sdd.SDD_E_CANCELLED
    t_b = time.perf_counter() - t0
    a.free()
    b.free()
    assert t_b < 0.1, t_b


def test_async_arguments():
    w = I.scaled(I.workload("quarterspace"), n_nodes=2, paths_per_node=100, dt=1e-3)
    ctx = sdd.sdd_create(w["model"])
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_interface_values_async(ctx, w["nodes"], w["n_paths"], w["dt"], 0, use_graph=1)
    assert e.value.status == sdd.SDD_E_UNSUPPORTED
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_interface_values_async(ctx, [[5.0, 0.0]], [10], w["dt"], 0)  # outside the domain
    assert e.value.status == sdd.SDD_E_ARG
    L = sdd.lib()
    assert L.sdd_poll(None) == sdd.SDD_E_ARG and L.sdd_wait(None, 0) == sdd.SDD_E_ARG

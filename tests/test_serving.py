"""The serving loop (sdd_server_*), through the C ABI.

Requests are random raster models shaped like the serving workload.  A
request's walks use the server seed and its node ids as Philox stream, so its
result must be the same whether it runs alone or batched with others (up to
the order of the FP64 sums), and the same as the single-model entry point.
"""
import time

import numpy as np
import pytest

from paper_1603_09311_gb300 import build as B
from paper_1603_09311_gb300 import inputs as I
from paper_1603_09311_gb300 import sdd

pytestmark = pytest.mark.gpu

DT, SEED = 1e-3, 4242
REL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    sdd.lib()


def _server(**kw):
    args = dict(domain=I.DOMAIN, nx=I.RASTER_NX, nz=I.RASTER_NZ, dt=DT, seed=SEED)
    args.update(kw)
    return sdd.Server(**args)


def _requests(n, seed=11, n_nodes=10):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        r = I.random_request(rng, i)
        nodes = r["nodes"][:: max(1, len(r["nodes"]) // n_nodes)][:n_nodes]
        r["nodes"] = nodes
        r["node_ids"] = np.arange(len(nodes)) + 1000 * i
        out.append(r)
    return out


def _spec(i):
    # even requests: fixed walk counts; odd ones: adaptive counts at a target SE
    if i % 2 == 0:
        return {"n_paths": 1500 + 100 * i}
    return {"target_se": 5e-3, "n_pilot": 512, "n_max": 40000}


def _run(srv, reqs, specs):
    ids = []
    for r, sp in zip(reqs, specs):
        rid = srv.submit(r["model"], r["nodes"], node_ids=r["node_ids"], **sp)
        assert rid is not None
        ids.append(rid)
    out = []
    for rid in ids:
        assert srv.wait(rid, 120_000)
        out.append(srv.result(rid))
    return out


def test_results_are_the_same_alone_and_in_the_mix():
    reqs = _requests(6)
    specs = [_spec(i) for i in range(len(reqs))]
    alone = _server(max_batch_models=1, n_streams=1)
    a = [_run(alone, [r], [sp])[0] for r, sp in zip(reqs, specs)]
    alone.close()
    mixed = _server(max_batch_models=64, n_streams=2)
    m = _run(mixed, reqs, specs)
    st = mixed.stats()
    mixed.close()
    assert st["completed"] == 6 and st["launches"] < 12  # batched: fewer launches than phases
    for (sa, ma, sea, ua, _), (sm, mm, sem, um, stm) in zip(a, m):
        assert sa == sm == sdd.SDD_OK
        assert np.array_equal(ua, um)
        scale = max(1.0, np.abs(ma).max())
        assert np.allclose(mm, ma, rtol=0, atol=REL * scale)
        assert np.allclose(sem, sea, rtol=1e-9, atol=0)
        assert stm["walks"] == ua.sum() and stm["latency_us"] > 0


def test_server_matches_the_single_model_entry_point():
    r = _requests(1, seed=3)[0]
    srv = _server()
    rid = srv.submit(r["model"], r["nodes"], n_paths=2500, node_ids=r["node_ids"])
    assert srv.wait(rid, 120_000)
    st, mean, se, used, stats = srv.result(rid)
    srv.close()
    ctx = sdd.sdd_create(r["model"])
    m1, s1, _ = sdd.sdd_interface_values(ctx, r["nodes"], 2500, DT, SEED, node_ids=r["node_ids"])
    assert st == sdd.SDD_OK and np.all(used == 2500)
    assert np.allclose(mean, m1, rtol=0, atol=REL * max(1.0, np.abs(m1).max()))
    assert np.allclose(se, s1, rtol=1e-9, atol=0)


def test_admission_refuses_beyond_slots_and_bytes():
    reqs = _requests(3, seed=5, n_nodes=4)
    srv = _server(max_requests=2)
    r0 = srv.submit(reqs[0]["model"], reqs[0]["nodes"], n_paths=200)
    r1 = srv.submit(reqs[1]["model"], reqs[1]["nodes"], n_paths=200)
    assert r0 is not None and r1 is not None
    assert srv.submit(reqs[2]["model"], reqs[2]["nodes"], n_paths=200) is None  # no slot
    assert srv.wait(r0, 60_000)
    srv.result(r0)  # frees a slot
    r2 = srv.submit(reqs[2]["model"], reqs[2]["nodes"], n_paths=200)
    assert r2 is not None
    for rid in (r1, r2):
        assert srv.wait(rid, 60_000)
        srv.result(rid)
    st = srv.stats()
    assert st["refused"] == 1 and st["in_flight"] == 0 and st["bytes_in_use"] == 0
    srv.close()
    # a byte budget smaller than one raster refuses everything
    tight = _server(max_bytes=1000)
    assert tight.submit(reqs[0]["model"], reqs[0]["nodes"], n_paths=10) is None
    tight.close()


def test_cancel_wait_timeout_and_unknown_ids():
    reqs = _requests(2, seed=9, n_nodes=64)
    srv = _server(n_streams=1, max_batch_models=1)
    big = srv.submit(reqs[0]["model"], reqs[0]["nodes"], n_paths=2_000_000)
    queued = srv.submit(reqs[1]["model"], reqs[1]["nodes"], n_paths=1000)
    time.sleep(0.01)
    srv.cancel(queued)  # still waiting behind the big request: ends at once
    assert srv.wait(queued, 1000)
    st, *_ = srv.result(queued)
    assert st == sdd.SDD_E_CANCELLED
    assert srv.wait(big, 1) is False  # a long request is not done after 1 ms
    assert srv.wait(big, -1) is True
    st, mean, se, used, stats = srv.result(big)
    # 64 nodes x 2e6 walks exceed the per-launch walk budget: the request ran in several pieces
    assert st == sdd.SDD_OK and np.all(np.isfinite(mean)) and stats["launches"] > 1
    with pytest.raises(sdd.SddError):
        srv.cancel(987654)
    with pytest.raises(sdd.SddError):
        srv.poll(987654)
    srv.close()


def test_a_small_request_overtakes_a_large_one_submitted_just_before():
    # one stream, launches of at most 2^20 walks: a large request (64 nodes x
    # 1e5 walks, 7 launches) and then a small one (16 nodes x 2000 walks).
    # Work is queued by virtual deadline (submission time + the phase's own
    # walk time), so the small request runs right after the large one's first
    # launch and ends first; queued by submission alone it would end last.
    rng = np.random.default_rng(21)
    big, small = I.random_request(rng, 0), I.random_request(rng, 1)
    big["nodes"] = np.resize(big["nodes"], (64, 2))
    small["nodes"] = small["nodes"][:16]
    srv = _server(n_streams=1, max_batch_models=1, max_batch_walks=1 << 20)
    rb = srv.submit(big["model"], big["nodes"], node_ids=np.arange(64), n_paths=100_000)
    rs = srv.submit(small["model"], small["nodes"], node_ids=np.arange(16) + 100, n_paths=2000)
    done = []
    t0 = time.perf_counter()
    while len(done) < 2 and time.perf_counter() - t0 < 120:
        for rid in (rb, rs):
            if rid not in done and srv.poll(rid):
                done.append(rid)
        time.sleep(0.0002)
    assert done == [rs, rb]
    assert srv.result(rs)[0] == sdd.SDD_OK and srv.result(rb)[0] == sdd.SDD_OK
    srv.close()

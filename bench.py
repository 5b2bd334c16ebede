"""Benchmark: TE Feynman-Kac interface-node Monte Carlo on one GB300.

One step = one full evaluation of the quarter-space workload: 64 interface
nodes on x = 0, z in [0, 0.9], 1e5 walks per node, dt = 1e-4 (dimensionless,
earth kappa 2 left / 20 right, air 0), single-precision walk with FP64 sums.

  value   walk-steps/s with the inputs resident in HBM (device-buffer C ABI,
          CUDA events on the launching stream, L2 flushed between steps)
  e2e     the same through the host-buffer C ABI (host<->device copies inside)
  roofline  issue-bound ("alu"): algorithmic thread-instructions per step x
          steps / walk-kernel time, against SMs x 128 lanes x max SM clock
  cpu_baseline  the FP64 oracle on the host cores, on a bounded sample

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) the ranks split one evaluation by (node, path-range)
units (shard.py): weak scaling (default) evaluates the 64 nodes with N x 1e5
walks each, strong scaling (--scaling strong) the 1e5 of one GPU's line.
Each rank walks a cost-balanced contiguous slice of the range list, one
all-reduce SUM of the zero-padded range-sum tables (NCCL) hands every rank
every range's sums, and each forms the node means in range order; rank 0
prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1603_09311_gb300 import inputs as I  # noqa: E402

WORKLOAD = "quarterspace"
METRIC = "walk-steps/s"
# Algorithmic thread-instructions per Euler step of the single-precision walk
# on the quarter-space model: half a Philox4x32-10
# call with the first round's fixed product precomputed (19.5), two uniforms
# from bit masks (3), Box-Muller (7), Euler update (2), wall distances and the
# bridge filter (5), the vertical-contact test as two compares (earth side,
# right of the contact) and one predicated add to each region counter (4),
# step bookkeeping (2.5).
INST_PER_STEP = 43
# The same count for a step of the TM walk (strips of their own diffusion):
# the TE step without its material test and counters (43 - 4), plus the
# interface tests (crossing compares 2, nearer interface product and filter
# 4) and the occupation update in shared memory (address and add, 2).
TM_INST_PER_STEP = 47
# The same count for the other lookup programs of the single-precision walk
# (the contact test's 4 replaced): one rectangle on one side of the surface
# (earth compare 1, four compares 4, two predicated region adds 2): 46; one
# triangle on one side of the surface (earth compare 1, three edge functions
# of two FMAs and a compare 9, two predicated region adds 2): 51.
RECT_INST_PER_STEP = 46
TRI_INST_PER_STEP = 51
# Walks per node of the double-precision leg of the triangle sweep.
FP64_WALKS = 50_000


def traffic_per_launch():
    """DRAM bytes per full walk launch from the last ncu capture in profiles/,
    or None when the kernel sources changed since that capture."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "walk_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    h = hashlib.sha256()
    for name in rec["kernel_source_files"]:
        with open(os.path.join(ROOT, name), "rb") as f:
            h.update(f.read())
    return rec["traffic_bytes_per_full_launch"] if h.hexdigest() == rec["kernel_source_sha256"] else None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi's own start-up stays outside the timed region: wait
            # (at most 3 s) for its first sample before the caller starts timing
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 3.0:
                time.sleep(0.01)
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def barrier_max(value: float, world: int, torch):
    if world == 1:
        return value
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(w, seconds_target: float = 15.0):
    """Time the oracle on a bounded sample of the workload: every node, the
    first n walks of each, n sized so the run takes about seconds_target."""
    from oracle import oracle as O
    threads = O.max_threads()
    probe = 100
    t0 = time.time()
    r = O.interface_values(w["model"], w["nodes"], probe, w["dt"], w["seed"], urule=23)
    dtp = max(time.time() - t0, 1e-3)
    n = int(min(max(probe, probe * seconds_target / dtp), w["n_paths"].max()))
    t0 = time.time()
    r = O.interface_values(w["model"], w["nodes"], n, w["dt"], w["seed"], urule=23)
    el = time.time() - t0
    return {"value": r["steps"] / el, "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": f"{len(w['nodes'])} nodes x first {n} walks of the workload "
                      f"({r['steps']:.3e} steps, {el:.1f} s)",
            "seconds": el}


def serving(sdd, n_requests: int, seed: int = 5, prefix: int = 200):
    """Serving run on the C5 request stream: random raster requests (16-1024
    nodes, target complex SE 1e-3, pilot 4096, cap 1e6 walks per node, dt 1e-3).
      - capacity: the server in closed loop (every request of the first
        `prefix` submitted at t = 0) against one request per launch on the
        same requests (the sum of their service times);
      - latency: all n_requests on Poisson arrivals at 0.7 x the capacity of
        one request per launch, served by the server (open loop), and the
        same arrivals served one request per launch in order (FIFO over the
        measured service times of every request)."""
    rng = np.random.default_rng(seed)
    reqs = [I.random_request(rng, i) for i in range(n_requests)]
    for r in reqs:
        r["node_ids"] = np.arange(len(r["nodes"]), dtype=np.uint32) + np.uint32(4096 * r["id"])
    kw = dict(target_se=1e-3, n_pilot=4096, n_max=1_000_000)

    def make_server():
        return sdd.Server(domain=I.DOMAIN, nx=I.RASTER_NX, nz=I.RASTER_NZ, dt=1e-3, seed=seed,
                          max_requests=64, n_streams=2, max_batch_models=64, max_batch_walks=1 << 25)

    def open_loop(srv, arrivals, reqs=reqs, kw=kw):
        t0 = time.perf_counter()
        pending, done_at, k = {}, {}, 0
        while len(done_at) < len(reqs):
            now = time.perf_counter() - t0
            while k < len(reqs) and arrivals[k] <= now:
                rid = srv.submit(reqs[k]["model"], reqs[k]["nodes"], node_ids=reqs[k]["node_ids"], **kw)
                if rid is None:
                    break  # no slot: retry on the next pass
                pending[rid] = k
                k += 1
            for rid in [r for r in pending if srv.poll(r)]:
                done_at[pending.pop(rid)] = time.perf_counter() - t0
                srv.result(rid)
            time.sleep(0.0002)
        lat = np.array([done_at[i] - arrivals[i] for i in range(len(reqs))])
        return lat, max(done_at.values())

    def fifo(arrivals, service):
        free_at, out = 0.0, []
        for a, s_ in zip(arrivals, service):
            free_at = max(a, free_at) + s_
            out.append(free_at - a)
        return np.array(out)

    # one request per launch: every request's service time (a request brings
    # its model: its upload is part of the service, as it is part of a served
    # request's latency)
    service, t_kernel = [], 0.0
    for r in reqs:
        t = time.perf_counter()
        ctx = sdd.sdd_create(r["model"])
        sdd.sdd_interface_values_target(ctx, r["nodes"], kw["n_pilot"], kw["n_max"], kw["target_se"],
                                        1e-3, seed, node_ids=r["node_ids"])
        ctx.close()
        service.append(time.perf_counter() - t)
    cap_base = len(reqs) / sum(service)
    # server capacity: closed loop over the prefix
    pre = reqs[:prefix]
    srv = make_server()
    st0 = srv.stats()
    _, span_c = open_loop(srv, np.zeros(len(pre)), pre)
    st1 = srv.stats()
    cap = len(pre) / span_c
    steps_c = st1["steps"] - st0["steps"]
    # latency: Poisson arrivals at 0.7 x the capacity of one request per launch
    arr = np.cumsum(np.random.default_rng(seed + 1).exponential(1.0 / (0.7 * cap_base), len(reqs)))
    arr -= arr[0]
    lat, span = open_loop(srv, arr)
    st2 = srv.stats()
    srv.close()
    base_lat = fifo(arr, service)
    # the plain form: one node per launch (pilot + top-up per node), on the
    # first requests only (it is far slower)
    n_plain = min(3, len(reqs))
    t_plain, nodes_plain = 0.0, 0
    for r in reqs[:n_plain]:
        ctx = sdd.sdd_create(r["model"])
        t = time.perf_counter()
        for j in range(len(r["nodes"])):
            sdd.sdd_interface_values_target(ctx, r["nodes"][j:j + 1], kw["n_pilot"], kw["n_max"],
                                            kw["target_se"], 1e-3, seed, node_ids=r["node_ids"][j:j + 1])
        t_plain += time.perf_counter() - t
        nodes_plain += len(r["nodes"])
        ctx.close()
    t_served = sum(service[:n_plain])
    total_nodes = sum(len(r["nodes"]) for r in reqs)

    # small requests (16-64 nodes, fixed 2e4 walks per node), where one
    # request alone cannot fill the GPU: closed-loop capacity of the server and
    # of one request per launch, then both on the same Poisson arrivals at
    # 0.7 x the capacity of one request per launch
    rng_s = np.random.default_rng(seed + 7)
    small = []
    for i in range(48):
        r = I.random_request(rng_s, 1000 + i)
        r["nodes"] = r["nodes"][: int(rng_s.integers(16, 65))]
        r["node_ids"] = np.arange(len(r["nodes"]), dtype=np.uint32) + np.uint32(4096 * r["id"])
        small.append(r)
    kw_s = dict(n_paths=20_000)
    srv = make_server()
    _, span_s = open_loop(srv, np.zeros(len(small)), small, kw_s)
    service_s = []
    for r in small:
        t = time.perf_counter()
        ctx = sdd.sdd_create(r["model"])
        sdd.sdd_interface_values(ctx, r["nodes"], kw_s["n_paths"], 1e-3, seed, node_ids=r["node_ids"])
        ctx.close()
        service_s.append(time.perf_counter() - t)
    cap_base_s = len(small) / sum(service_s)
    arr_s = np.cumsum(np.random.default_rng(seed + 8).exponential(1.0 / (0.7 * cap_base_s), len(small)))
    arr_s -= arr_s[0]
    lat_s, _ = open_loop(srv, arr_s, small, kw_s)
    srv.close()
    base_s = fifo(arr_s, service_s)
    small_out = {
        "requests": len(small), "workload": "random raster requests, 16-64 nodes, 2e4 walks per node, dt 1e-3",
        "arrivals": "Poisson at 0.7 x the capacity of one request per launch",
        "capacity_req_per_s": len(small) / span_s,
        "p50_ms": 1e3 * float(np.percentile(lat_s, 50)), "p99_ms": 1e3 * float(np.percentile(lat_s, 99)),
        "baseline_one_request_per_launch": {
            "capacity_req_per_s": cap_base_s,
            "p50_ms": 1e3 * float(np.percentile(base_s, 50)),
            "p99_ms": 1e3 * float(np.percentile(base_s, 99))}}
    return {"requests": len(reqs),
            "capacity_req_per_s": cap, "capacity_requests": len(pre),
            "capacity_steps_per_s": steps_c / span_c,
            "baseline_capacity_same_requests": len(pre) / sum(service[:len(pre)]),
            "capacity_gain": cap / (len(pre) / sum(service[:len(pre)])),
            "arrivals": "Poisson at 0.7 x the capacity of one request per launch (all requests)",
            "arrival_rate_req_per_s": 0.7 * cap_base,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "steps_per_s": (st2["steps"] - st1["steps"]) / span,
            "launches": int(st2["launches"] - st0["launches"]),
            "node_solves_per_s": total_nodes / span,
            "baseline_one_request_per_launch": {
                "capacity_req_per_s": cap_base,
                "p50_ms": 1e3 * float(np.percentile(base_lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(base_lat, 99))},
            "baseline_one_node_per_launch": {
                "requests": n_plain, "nodes": nodes_plain,
                "node_solves_per_s": nodes_plain / t_plain,
                "slowdown_vs_one_request_per_launch": t_plain / t_served},
            "workload": "random raster requests (1024x768 int8, 1-4 shapes), 16-1024 nodes, "
                        "target SE 1e-3, pilot 4096, cap 1e6, dt 1e-3",
            "server": "2 streams, up to 2^25 walks and 64 models per launch",
            "small_requests": small_out}


def tm_measure(sdd, torch, dev, peak_tinst, n_steps, cpu=True, tune=True):
    """The TM walk on the analytic test model's 51 x 51 grid (2401 nodes x 1e4
    walks, dt 1e-4): walk-steps/s of the device entry point (CUDA events on the
    launching stream, L2 flushed between launches), its issue roofline, and
    the oracle on the host cores on a bounded sample."""
    w = I.workload("tm_analytic")
    n = len(w["nodes"])
    ctx = sdd.sdd_create(w["model"])
    shape = tune_shape(sdd, ctx, w, w["dt"]) if tune else "default shape"
    d_nodes = torch.tensor(w["nodes"], dtype=torch.float64, device=dev)
    d_mean = torch.empty((n, ctx.E, 2), dtype=torch.float64, device=dev)
    d_se = torch.empty_like(d_mean)
    d_cnt = torch.zeros((n_steps + 1, 3), dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def launch(k):
        sdd.sdd_interface_values_device(ctx, d_nodes.data_ptr(), n, w["n_paths"], w["dt"], w["seed"] + k,
                                        d_mean.data_ptr(), d_se.data_ptr(), d_counters_ptr=d_cnt[k].data_ptr(),
                                        stream=stream.cuda_stream)

    launch(n_steps)  # warm-up
    torch.cuda.synchronize()
    ms = []
    for k in range(n_steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        launch(k)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    steps = d_cnt[:n_steps, 0].cpu().numpy().astype(float)
    value = float(steps.sum() / (sum(ms) * 1e-3))
    out = {"metric": METRIC, "value": value, "unit": METRIC, "ms_per_launch": statistics.mean(ms),
           "launches": n_steps, "steps_per_launch": float(steps.mean()),
           "workload": "TM analytic test model: [-1,1]^2, D 1|10 across x=0, kappa -10 (lambda 10i), "
                       "2401 nodes (51x51 grid interior) x 1e4 walks, dt 1e-4, FP32 walk",
           "launch": shape,
           "roofline": {"bound": "alu", "achieved": TM_INST_PER_STEP * value / 1e12, "peak": peak_tinst,
                        "unit": "Tinst/s", "frac": TM_INST_PER_STEP * value / 1e12 / peak_tinst,
                        "inst_per_step": TM_INST_PER_STEP}}
    if cpu:
        # the FP32 TM walk against the oracle on the same streams: every 100th
        # node (25 nodes across the grid) under its own node id, first 2000
        # walks; the oracle's timing of that sample is the baseline
        out["fp32_error"], out["cpu_baseline"] = fp32_error(sdd, ctx, w, np.arange(0, n, 100), 2000,
                                                            w["dt"], w["seed"])
    ctx.close()
    return out


def device_launches(sdd, torch, dev, ctx, w, dt, seeds, flush, precision="fp32"):
    """Device-buffer launches of a workload, one per seed, L2 flushed before
    each; CUDA events on the launching stream.  Returns (ms per launch,
    steps per launch, walks per launch)."""
    n = len(w["nodes"])
    d_nodes = torch.tensor(w["nodes"], dtype=torch.float64, device=dev)
    d_ids = torch.arange(n, dtype=torch.int32, device=dev)
    d_mean = torch.empty((n, ctx.E, 2), dtype=torch.float64, device=dev)
    d_se = torch.empty_like(d_mean)
    d_cnt = torch.zeros((len(seeds), 3), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    evs = []
    for k, sd in enumerate(seeds):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sdd.sdd_interface_values_device(ctx, d_nodes.data_ptr(), n, w["n_paths"], dt, sd, d_mean.data_ptr(),
                                        d_se.data_ptr(), d_node_ids_ptr=d_ids.data_ptr(),
                                        d_counters_ptr=d_cnt[k].data_ptr(), stream=stream.cuda_stream,
                                        precision=precision)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    cnt = d_cnt.cpu().numpy()
    return [a.elapsed_time(b) for a, b in evs], cnt[:, 0].astype(float), cnt[:, 1].astype(float)


def _dev_stats(d):
    """Largest and rms of |d| (an array of deviations)."""
    d = np.abs(np.asarray(d, dtype=float)).ravel()
    return {"max": float(d.max()), "rms": float(np.sqrt((d ** 2).mean()))}


def fp32_error(sdd, ctx, w, idx, n_sub, dt, seed, ref_cache=None):
    """The single-precision walk against the FP64 oracle on the same random
    streams: nodes idx under their own node ids, the first n_sub walks of
    each, the oracle with the same 23-bit uniform rule.  Returns |GPU -
    oracle| (absolute, and in units of the oracle's standard error) over
    every node, evaluation and component, and the oracle's own timing."""
    from oracle import oracle as O
    idx = [int(j) for j in idx]
    nodes = w["nodes"][idx]
    m32, s32, st = sdd.sdd_interface_values(ctx, nodes, n_sub, dt, seed,
                                            node_ids=np.asarray(idx, dtype=np.uint32))
    t = time.perf_counter()
    ref, ref_se, steps = [], [], 0
    for j in idx:
        r = O.interface_values(w["model"], w["nodes"][j:j + 1], n_sub, dt, seed, urule=23, node_id0=j)
        ref.append(r["mean"][0])
        ref_se.append(r["se"][0])
        steps += r["steps"]
    sec = time.perf_counter() - t
    ref, ref_se = np.array(ref), np.array(ref_se)
    d = m32 - ref
    d2 = np.stack([d.real, d.imag], axis=-1)
    out = {"nodes": idx, "walks_per_node": int(n_sub), "dt": dt, "streams": "same (23-bit uniform rule)",
           "abs": _dev_stats(d2), "in_se": _dev_stats(d2 / ref_se),
           "se_median": float(np.median(ref_se)),
           "step_totals": {"gpu": int(st["steps"]), "oracle": int(steps)}}
    return out, {"value": steps / sec, "unit": METRIC, "cores": O.max_threads(), "kind": "oracle",
                 "sample": f"nodes {idx} x first {n_sub} walks, dt {dt} ({steps:.3e} steps, {sec:.1f} s)"}


def tune_shape(sdd, ctx, w, dt):
    """The launch shape for a workload, searched on w (untimed; the context
    keeps the fastest, as the main line's does)."""
    cfg, rate = sdd.sdd_autotune(ctx, w["nodes"], w["n_paths"], dt, w["seed"] + 999)
    return dict(cfg, walk_steps_per_s_while_tuning=rate)


def block_measure(sdd, torch, dev, peak_tinst, flush, reps=2, cpu=True, tune=True):
    """The batched block workload in full: 256 nodes on the perimeter of the
    block [-0.2,0.2]x[0.2,0.5] (rates 20 and 0.2 in host 2, x 8 frequency
    scales = 16 evaluations per walk), walks per node log-uniform in
    [1e4, 1e6] (5.5e7 walks), dt 1e-4, one launch; walk-steps/s of the
    device entry point and its issue roofline."""
    w = I.workload("block")
    ctx = sdd.sdd_create(w["model"])
    sdd.sdd_interface_values(ctx, w["nodes"][:4], 2000, w["dt"], 1)  # loads the kernel
    # shape searched on 64 of the nodes with their walk counts
    shape = tune_shape(sdd, ctx, I.scaled(w, n_nodes=64), w["dt"]) if tune else "default shape"
    ms, steps, walks = device_launches(sdd, torch, dev, ctx, w, w["dt"],
                                       [w["seed"] + k for k in range(reps)], flush)
    value = float(steps.sum() / (sum(ms) * 1e-3))
    ach = RECT_INST_PER_STEP * value / 1e12
    out = {"metric": METRIC, "value": value, "unit": METRIC, "ms_per_launch": statistics.mean(ms),
           "launches": reps, "steps_per_launch": float(steps.mean()), "walks_per_launch": float(walks.mean()),
           "workload": "block in half-space: 256 perimeter nodes, 1e4-1e6 walks per node (log-uniform, "
                       "seed 3), 16 evaluations per walk (rates 20 | 0.2 x 8 scales 0.1-100), dt 1e-4, "
                       "one launch, FP32 walk, FP64 sums",
           "launch": shape,
           "roofline": {"bound": "alu", "achieved": ach, "peak": peak_tinst, "unit": "Tinst/s",
                        "frac": ach / peak_tinst, "inst_per_step": RECT_INST_PER_STEP}}
    if cpu:
        # the four nodes with the fewest walks, their first 20000 walks
        idx = np.argsort(w["n_paths"])[:4]
        out["fp32_error"], out["cpu_baseline"] = fp32_error(sdd, ctx, w, idx, 20000, w["dt"], w["seed"])
    ctx.close()
    return out


def triangle_measure(sdd, torch, dev, peak_tinst, flush, cpu=True, tune=True):
    """The triangle time-step sweep in full: 128 nodes on the edges of the
    triangle (-0.3,0.2),(0.3,0.2),(0,0.6) (rate 50 in host 2), 1e6 walks per
    node, dt in {1e-3, 3e-4, 1e-4, 3e-5}, one FP32 launch per dt; the FP64
    walk on four of the nodes at each dt (its own 32-bit uniform stream), and
    the FP32 error against the oracle on the same streams."""
    w = I.workload("triangle")
    ctx = sdd.sdd_create(w["model"])
    sdd.sdd_interface_values(ctx, w["nodes"][:4], 2000, 1e-3, 1)
    # one shape for the sweep, searched at dt 1e-4 on 2e5 walks per node
    shape = tune_shape(sdd, ctx, I.scaled(w, paths_per_node=200_000), 1e-4) if tune else "default shape"
    sub = [0, 40, 85, 127]
    per_dt, tot_steps, tot_ms = [], 0.0, 0.0
    for dt in (1e-3, 3e-4, 1e-4, 3e-5):
        ms, steps, walks = device_launches(sdd, torch, dev, ctx, w, dt, [w["seed"]], flush)
        m32, s32, _ = sdd.sdd_interface_values(ctx, w["nodes"][sub], w["n_paths"][sub], dt, w["seed"],
                                               node_ids=np.asarray(sub, dtype=np.uint32))
        t = time.perf_counter()
        m64, s64, st64 = sdd.sdd_interface_values(ctx, w["nodes"][sub], FP64_WALKS, dt, w["seed"],
                                                  node_ids=np.asarray(sub, dtype=np.uint32), precision="fp64")
        t64 = time.perf_counter() - t
        d = m32 - m64
        cse = np.sqrt(s32 ** 2 + s64 ** 2)
        d2 = np.stack([d.real, d.imag], axis=-1)
        v = float(steps[0] / (ms[0] * 1e-3))
        ent = {"dt": dt, "value": v, "ms": ms[0], "steps": float(steps[0]), "walks": float(walks[0]),
               "frac": TRI_INST_PER_STEP * v / 1e12 / peak_tinst,
               "fp32_vs_gpu_fp64": {"nodes": sub, "walks_fp32": 1_000_000, "walks_fp64": FP64_WALKS,
                                    "streams": "independent (23- and 32-bit uniform rules)",
                                    "abs": _dev_stats(d2), "in_combined_se": _dev_stats(d2 / cse),
                                    "fp64_steps_per_s": st64["steps"] / (st64["kernel_ms"] * 1e-3),
                                    "fp64_seconds": t64}}
        if cpu:
            n_sub = int(min(100_000, max(2000, 6e7 / (0.4 / dt) / 2)))
            ent["fp32_error"], ent["cpu_baseline"] = fp32_error(sdd, ctx, w, [40, 85], n_sub, dt, w["seed"])
        per_dt.append(ent)
        tot_steps += steps[0]
        tot_ms += ms[0]
    ctx.close()
    value = tot_steps / (tot_ms * 1e-3)
    ach = TRI_INST_PER_STEP * value / 1e12
    return {"metric": METRIC, "value": value, "unit": METRIC, "ms": tot_ms, "steps": tot_steps,
            "workload": "triangle in half-space: 128 edge nodes x 1e6 walks, rate 50 in host 2, "
                        "dt 1e-3, 3e-4, 1e-4, 3e-5 (one launch each), FP32 walk, FP64 sums",
            "launch": shape,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak_tinst, "unit": "Tinst/s",
                         "frac": ach / peak_tinst, "inst_per_step": TRI_INST_PER_STEP},
            "per_dt": per_dt}


def small_cases(sdd, objs):
    """Two launches of a small case of the block and/or triangle workloads
    through the host-buffer entry point: walk-steps/s of the second."""
    out = {}
    if "block" in objs:
        w = I.workload("block")
        idx = np.arange(0, 256, 4)
        ctx = sdd.sdd_create(w["model"])
        npth = np.maximum(w["n_paths"][idx] // 8, 1000)
        for k in range(2):
            _, _, st = sdd.sdd_interface_values(ctx, w["nodes"][idx], npth, w["dt"], w["seed"] + k,
                                                node_ids=idx.astype(np.uint32))
        out["block"] = {"steps": st["steps"], "value": st["steps"] / (st["kernel_ms"] * 1e-3),
                        "workload": "64 of the block workload's nodes (every 4th), 1/8 of their walks"}
        ctx.close()
    if "triangle" in objs:
        t = I.scaled(I.workload("triangle"), n_nodes=16, paths_per_node=100_000)
        ctx = sdd.sdd_create(t["model"])
        for k in range(2):
            _, _, st = sdd.sdd_interface_values(ctx, t["nodes"], t["n_paths"], t["dt"], t["seed"] + k)
        out["triangle"] = {"steps": st["steps"], "value": st["steps"] / (st["kernel_ms"] * 1e-3),
                           "workload": "16 of the triangle workload's nodes x 1e5 walks, dt 1e-4"}
        ctx.close()
    return out


def interp_measure(sdd, reps=3, cpu=True):
    """Interpolation along an interface (Sec. 5): the quarter-space line of 64
    nodes at 1e5 walks per walked node, walks at every 4th node and the last
    (17 of 64), the others interpolated in arc length; against walks at all 64
    nodes.  Host-buffer calls timed end to end (wall clock, best of reps), the
    interpolation kernels by CUDA events inside the call.  The deviation of
    an interpolated node from its own walks is given in units of their
    combined standard error."""
    w = I.workload("quarterspace")
    nodes, n = w["nodes"], len(w["nodes"])
    stride, paths = 4, int(w["n_paths"][0])
    knots = list(range(0, n, stride))
    if knots[-1] != n - 1:
        knots.append(n - 1)
    ctx = sdd.sdd_create(w["model"])
    ids = np.arange(n, dtype=np.uint32)

    def best(f):
        out, t_best = None, float("inf")
        for _ in range(reps):
            t = time.perf_counter()
            r = f()
            t_best = min(t_best, time.perf_counter() - t)
            out = r
        return out, t_best

    sdd.sdd_interface_values(ctx, nodes, paths, w["dt"], w["seed"], node_ids=ids)  # warm-up
    (full, fse, fst), t_full = best(lambda: sdd.sdd_interface_values(ctx, nodes, paths, w["dt"], w["seed"],
                                                                     node_ids=ids))
    skip = np.setdiff1d(np.arange(n), knots)
    out = {"workload": (f"quarterspace line: {n} nodes on x=0, z in [0,0.9], {paths} walks per walked "
                        f"node, dt 1e-4; walks at every {stride}th node and the last ({len(knots)} of {n}), "
                        "the others interpolated in arc length"),
           "unit": "interface-node values/s", "full": {"value": n / t_full, "ms": 1e3 * t_full,
                                                      "walk_kernel_ms": fst["kernel_ms"]}}
    for name, kind in (("spline", sdd.SDD_INTERP_SPLINE), ("linear", sdd.SDD_INTERP_LINEAR)):
        sdd.sdd_interface_values_interp(ctx, nodes, stride, paths, kind, w["dt"], w["seed"])
        (m, se, st), t = best(lambda: sdd.sdd_interface_values_interp(ctx, nodes, stride, paths, kind,
                                                                      w["dt"], w["seed"]))
        zr = np.abs(m[skip].real - full[skip].real) / np.sqrt(se[skip, :, 0] ** 2 + fse[skip, :, 0] ** 2)
        zi = np.abs(m[skip].imag - full[skip].imag) / np.sqrt(se[skip, :, 1] ** 2 + fse[skip, :, 1] ** 2)
        z = np.concatenate([zr.ravel(), zi.ravel()])
        out[name] = {"value": n / t, "ms": 1e3 * t, "speedup": t_full / t, "walks": int(st["walks"]),
                     "walk_kernel_ms": st["kernel_ms"], "interp_kernel_ms": st["post_ms"],
                     "interp_launches": int(st["launches"]) - 2,
                     "max_dev_in_se": float(z.max()), "rms_dev_in_se": float(np.sqrt((z ** 2).mean()))}
    out["value"] = out["spline"]["value"]
    out["fp32_error"] = "the walks at the knots are the main line's kernel and model: its fp32_error"
    out["roofline"] = {"bound": "latency",
                       "note": "the interpolation kernels move a few KB in a few launches of microseconds; "
                               "the walks at the knots are the time, bounded as the main line's kernel"}
    ctx.close()
    if cpu:
        from oracle import interp as OI
        s = OI.arc_length(nodes)
        kv = np.stack([full[knots].real, full[knots].imag], axis=-1).reshape(len(knots), -1)
        ke = fse[knots].reshape(len(knots), -1)
        t = time.perf_counter()
        k = 0
        while time.perf_counter() - t < 1.0:
            OI.interpolate(s[knots], kv, ke, s, OI.SPLINE)
            k += 1
        sec = (time.perf_counter() - t) / k
        out["cpu_baseline"] = {"value": n / sec, "unit": "interface-node values/s (interpolation only)",
                               "cores": 1, "kind": "oracle",
                               "sample": f"the spline interpolation of the {len(knots)} knots to {n} nodes, "
                                         f"{k} repetitions ({1e3 * sec:.2f} ms each)"}
    return out


def mt_measure(sdd, reps=3, cpu=True):
    """Apparent resistivity and phase at measurement sites (Sec. 2.1, Sec.
    4.2): the block-in-half-space model (16 evaluations: two block rates x 8
    frequency scales), 5 surface sites, three points each 0.02 apart
    straddling the surface, 4e5 walks per point (the paper's N = 400 000),
    dt 1e-4.  Host-buffer call timed end to end (best of reps)."""
    w = I.workload("block")
    model = w["model"]
    kref = np.asarray(model["kappa"])[:, 1]  # the host rock as reference
    sites = np.array([[0.0, 0.0], [0.1, 0.0], [0.2, 0.0], [0.4, 0.0], [0.8, 0.0]])
    h, paths, dt, seed = 0.02, 400_000, 1e-4, 41
    ctx = sdd.sdd_create(model)
    r = sdd.sdd_apparent_resistivity(ctx, sites, h, paths, kref, dt, seed)  # warm-up
    t_best = float("inf")
    for _ in range(reps):
        t = time.perf_counter()
        r = sdd.sdd_apparent_resistivity(ctx, sites, h, paths, kref, dt, seed)
        t_best = min(t_best, time.perf_counter() - t)
    ctx.close()
    st = r["stats"]
    n_out = r["rho"].size
    out = {"workload": (f"block in half-space, {r['rho'].shape[1]} evaluations, sites x in "
                        f"{sites[:, 0].tolist()} on the surface, 3 points h = {h} apart, {paths} walks per "
                        f"point, dt {dt}; rho in units of the host rock's resistivity"),
           "value": n_out / t_best, "unit": "site-evaluation (rho, phi) values/s", "ms": 1e3 * t_best,
           "walks": int(st["walks"]), "steps": int(st["steps"]), "walk_kernel_ms": st["kernel_ms"],
           "walk_steps_per_s": st["steps"] / (st["kernel_ms"] * 1e-3), "post_kernel_ms": st["post_ms"],
           "rel_rho_se_median": float(np.median(r["rho_se"] / r["rho"])),
           "phase_se_median_deg": float(np.degrees(np.median(r["phase_se"]))),
           "rho_site0": [round(float(v), 4) for v in r["rho"][0, :8]],
           "fp32_error": "the walks at the three points are the block object's kernel and model: its fp32_error",
           "roofline": {"bound": "alu", "note": "the walks of the 15 points (the main line's kernel) are the "
                                                "time; the resistivity kernel is one launch of microseconds"}}
    if cpu:
        from oracle import oracle as O
        from oracle import mt as OM
        sample = 4000
        t = time.perf_counter()
        pts = OM.site_points(sites[:1], h)
        O.interface_values(model, pts, sample, dt, seed, urule=23)
        sec = (time.perf_counter() - t) * paths / sample
        out["cpu_baseline"] = {"value": r["rho"].shape[1] / sec, "unit": out["unit"], "cores": O.max_threads(),
                               "kind": "oracle",
                               "sample": f"one site's 3 points x {sample} walks, scaled to {paths} walks"}
    return out


def rbffd_measure(sdd, reps=2, cpu=True):
    """The stochastic domain decomposition end to end (Sec. 3): sub-domain
    [0, 0.9]^2 of the quarter-space model (rate 20 inside, bounded by the
    air-earth interface and the vertical contact), walks at its 720 boundary
    nodes (1e5 walks each, dt 1e-4), then the RBF-FD solve (Sec. 3.2: 9-node
    multiquadric stencils, eps 1) at its 32041 inner nodes of a 181 x 181
    grid, eps 5 (eps h = 0.025; the paper's eps h is about 0.05).  Host-buffer
    calls timed end to end (best of reps)."""
    w = I.workload("quarterspace")
    n_side = 181
    nodes, edge = I.rect_grid(0, 0.9, 0, 0.9, n_side, n_side)
    bnd = np.flatnonzero(edge == 1)
    paths, dt, seed = 100_000, 1e-4, 61
    kap = np.full(len(nodes), 20.0)
    eps = 5.0
    ctx = sdd.sdd_create(w["model"])

    def run():
        t0 = time.perf_counter()
        m, se, st = sdd.sdd_interface_values(ctx, nodes[bnd], paths, dt, seed)
        t1 = time.perf_counter()
        vals = np.zeros(len(nodes), dtype=complex)
        vals[bnd] = m[:, 0]
        u, rs = sdd.sdd_rbffd_solve(nodes, edge, vals, kap, 9, eps, tol=1e-10)
        t2 = time.perf_counter()
        return t1 - t0, t2 - t1, st, rs

    run()  # warm-up
    best = None
    for _ in range(reps):
        r = run()
        if best is None or r[0] + r[1] < best[0] + best[1]:
            best = r
    ctx.close()
    t_mc, t_rb, st, rs = best
    out = {"workload": (f"quarter-space sub-domain [0,0.9]^2: walks at {len(bnd)} boundary nodes ({paths} each, "
                        f"dt {dt}), RBF-FD (9-node multiquadric, eps 5) at {rs['unknowns']} inner nodes of "
                        f"a {n_side} x {n_side} grid, BiCGStab to 1e-10"),
           "value": len(nodes) / (t_mc + t_rb), "unit": "sub-domain node values/s (walks + RBF-FD)",
           "ms": 1e3 * (t_mc + t_rb), "walks_ms": 1e3 * t_mc, "walk_kernel_ms": st["kernel_ms"],
           "rbffd_ms": 1e3 * t_rb, "knn_kernel_ms": rs["knn_ms"], "weights_kernel_ms": rs["weights_ms"],
           "solve_ms": rs["solve_ms"], "iterations": rs["iterations"], "rel_residual": rs["rel_residual"],
           "ms_per_iteration": rs["solve_ms"] / max(rs["iterations"], 1),
           "fp32_error": "the boundary walks are the main line's kernel and model: its fp32_error; "
                         "the RBF-FD stage is FP64",
           "roofline": {"bound": "latency",
                        "note": "a BiCGStab iteration is 5 launches (replayed 8 iterations at a time as a "
                                "CUDA graph) over vectors of 32k complex values (a few MB, L2-resident); the "
                                "walks at the boundary nodes are bounded as the main line's kernel"}}
    if cpu:
        from oracle import rbffd as R
        sn, se_ = I.rect_grid(0, 0.9, 0, 0.9, 37, 37)
        vals = np.where(se_ == 1, 1.0 + 0.0j, 0.0)
        t = time.perf_counter()
        R.solve(sn, se_, vals, np.full(len(sn), 20.0), 9, 5.0)
        sec = time.perf_counter() - t
        out["cpu_baseline"] = {"value": len(sn) / sec, "unit": "sub-domain node values/s (RBF-FD only)",
                               "cores": 1, "kind": "oracle",
                               "sample": f"the RBF-FD stage on a 37 x 37 grid of the same sub-domain "
                                         f"({len(sn)} nodes, {sec:.2f} s)"}
    return out


def run_sharded(args, torch, rank, world, local):
    """The quarter-space evaluation split across `world` ranks (one GPU each)
    by (node, path-range) units; timed per step from the first range launch
    to the node means, max over ranks."""
    import torch.distributed as dist
    from paper_1603_09311_gb300 import sdd
    from paper_1603_09311_gb300 import shard as S
    w = I.workload(WORKLOAD)
    n = len(w["nodes"])
    per_node = int(w["n_paths"][0]) * (world if args.scaling == "weak" else 1)
    npth = np.full(n, per_node, dtype=np.int64)
    P = S.plan(w["nodes"], npth, args.chunk, world, I.DOMAIN)
    b, e = int(P["bounds"][rank]), int(P["bounds"][rank + 1])
    node, begin, count = P["node"], P["begin"], P["count"]
    m = len(node)
    dev = torch.device("cuda", local)
    ctx = sdd.sdd_create(w["model"])
    d_nodes = torch.tensor(w["nodes"][node[b:e]], dtype=torch.float64, device=dev).reshape(-1, 2)
    d_ids = torch.tensor(node[b:e].astype(np.int32), device=dev)
    table = torch.zeros((m, ctx.E, 4), dtype=torch.float64, device=dev)
    nvalid = torch.zeros(m, dtype=torch.int64, device=dev)
    d_mean = torch.empty((n, ctx.E, 2), dtype=torch.float64, device=dev)
    d_se = torch.empty_like(d_mean)
    d_cnt = torch.zeros((max(args.steps, args.warmup), 3), dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(seed, k):
        # rows of the other ranks are zero before the all-reduce
        table[:b].zero_()
        table[e:].zero_()
        nvalid[:b].zero_()
        nvalid[e:].zero_()
        if e > b:
            sdd.sdd_range_sums_device(ctx, d_nodes.data_ptr(), e - b, begin[b:e], count[b:e], w["dt"], seed,
                                      table[b:e].data_ptr(), nvalid[b:e].data_ptr(),
                                      d_node_ids_ptr=d_ids.data_ptr(), d_counters_ptr=d_cnt[k].data_ptr(),
                                      stream=stream.cuda_stream)
        S.allreduce_table(table, dist)
        S.allreduce_table(nvalid, dist)
        sdd.sdd_reduce_sums_device(ctx, n, node, table.data_ptr(), nvalid.data_ptr(), d_mean.data_ptr(),
                                   d_se.data_ptr(), stream=stream.cuda_stream)

    for i in range(args.warmup):
        step(w["seed"] + 1000 + i, i)
    torch.cuda.synchronize()
    d_cnt.zero_()
    sampler = ClockSampler(local)
    sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        step(w["seed"] + k, k)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clocks = sampler.stop()
    total_ms = barrier_max(sum(a.elapsed_time(b_) for a, b_ in evs), world, torch)
    steps_local = torch.tensor([float(d_cnt[: args.steps, 0].sum())], dtype=torch.float64, device=dev)
    dist.all_reduce(steps_local)  # every rank's walk-steps
    steps_all = float(steps_local.item())
    walks = int(nvalid.sum())
    assert walks == n * per_node, "a step did not reach every walk"
    value = steps_all / (total_ms * 1e-3)
    peaks, src = load_peaks()
    clk_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tinst = world * n_sm * 128 * clk_mhz * 1e6 / 1e12
    achieved = INST_PER_STEP * value / 1e12
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": args.scaling, "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": (f"quarterspace: {n} nodes on x=0, z in [0,0.9], {per_node} walks/node, "
                                    "dt 1e-4, kappa 2|20 earth, 0 air (dimensionless)"),
                       "parallelism": (f"{world} ranks x (node, path-range) slices of {args.chunk}-walk ranges "
                                       f"({m} ranges, balanced by expected steps), one NCCL all-reduce of the "
                                       "zero-padded range-sum table per step, node means in range order"),
                       "walks_per_step": n * per_node, "l2": "flushed between steps (256 MB write)",
                       "precision": "FP32 walk, FP64 sums"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tinst, "unit": "Tinst/s",
                         "frac": achieved / peak_tinst, "inst_per_step": INST_PER_STEP,
                         "peak_source": f"{world} GPUs x {n_sm} SMs x 128 lanes x {clk_mhz:.0f} MHz ({src})"},
            "clocks": clocks, "gpu_launches": 3 * args.steps,
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                    "note": "multi-rank steps are device-resident; the host-buffer form is measured at N = 1"},
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    dist.destroy_process_group()
    return 0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = I.workload(WORKLOAD)
    from oracle import oracle as O
    # each step: every node, a bounded number of walks, sized so the whole run
    # (warmup + steps) ends within a few minutes
    total_steps = args.warmup + args.steps
    per_step_s = max(2.0, 150.0 / total_steps)
    base = cpu_baseline(w, per_step_s)
    n = int(base["sample"].split("first ")[1].split(" ")[0])
    times, steps = [], 0
    for i in range(total_steps):
        t0 = time.time()
        r = O.interface_values(w["model"], w["nodes"], n, w["dt"], w["seed"] + i, urule=23)
        el = time.time() - t0
        if i >= args.warmup:
            times.append(el)
            steps += r["steps"]
    value = steps / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: 64 nodes, first {n} of 1e5 walks per node, dt 1e-4",
                       "l2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": base["cores"],
                             "kind": "oracle", "sample": f"64 nodes x {n} walks per step"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sdd", choices=["sdd", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--graph", action="store_true", help="run each step as a CUDA graph")
    ap.add_argument("--serve-requests", type=int, default=400,
                    help="requests of the serving measurement (0 skips it)")
    ap.add_argument("--small", action="store_true",
                    help="16 nodes x 1e5 walks of the same workload (for profiler captures)")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="N > 1: weak = N x 1e5 walks per node split across the ranks, strong = 1e5")
    ap.add_argument("--chunk", type=int, default=4096, help="N > 1: walks per (node, path-range) unit")
    ap.add_argument("--sharded", action="store_true",
                    help="run the multi-rank form (range sums, all-reduce, reduction) even at N = 1")
    ap.add_argument("--objects", default="all",
                    help="comma-separated objects added to the line: serving, tm, interp, mt, rbffd, "
                         "block, triangle (default all)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1 or args.sharded:
        import torch.distributed as dist
        if not dist.is_initialized():
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            os.environ.setdefault("MASTER_PORT", "29531")
            dist.init_process_group("nccl", device_id=torch.device("cuda", local), rank=rank, world_size=world)
    from paper_1603_09311_gb300 import build as B
    from paper_1603_09311_gb300 import sdd
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    B.build()
    if world > 1 or args.sharded:
        return run_sharded(args, torch, rank, world, local)

    w = I.workload(WORKLOAD)
    if args.small:
        w = I.scaled(w, n_nodes=16)
    n = len(w["nodes"])
    node_ids = np.arange(n, dtype=np.uint32)
    ctx = sdd.sdd_create(w["model"])
    dev = torch.device("cuda", local)
    d_nodes = torch.tensor(w["nodes"], dtype=torch.float64, device=dev)
    d_ids = torch.tensor(node_ids.astype(np.int64), dtype=torch.int64, device=dev).to(torch.int32)
    d_mean = torch.empty((n, ctx.E, 2), dtype=torch.float64, device=dev)
    d_se = torch.empty((n, ctx.E, 2), dtype=torch.float64, device=dev)
    d_cnt = torch.zeros((max(args.steps, args.warmup), 3), dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step(seed, k):
        sdd.sdd_interface_values_device(ctx, d_nodes.data_ptr(), n, w["n_paths"], w["dt"], seed,
                                        d_mean.data_ptr(), d_se.data_ptr(),
                                        d_node_ids_ptr=d_ids.data_ptr(),
                                        d_counters_ptr=d_cnt[k].data_ptr(), stream=stream.cuda_stream,
                                        use_graph=int(args.graph))

    tuned = None
    if not args.no_autotune:
        # launch shape for this workload (untimed; the context keeps it)
        cfg_t, rate_t = sdd.sdd_autotune(ctx, w["nodes"], w["n_paths"], w["dt"], w["seed"] + 999)
        tuned = dict(cfg_t, walk_steps_per_s=rate_t)
    for i in range(args.warmup):
        step(w["seed"] + 1000 + i, i)
    torch.cuda.synchronize()

    # ---- device-resident timed region: K steps, L2 flushed between steps
    sampler = ClockSampler(local)
    sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        step(w["seed"] + k, k)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    cnt = d_cnt[: args.steps].cpu().numpy()
    steps_local = int(cnt[:, 0].sum())
    steps_done_one = steps_local / args.steps
    assert int(cnt[:, 1].min()) == n * int(w["n_paths"][0]), "a step did not run every walk"
    steps_done = steps_local
    mean = d_mean.cpu().numpy()
    se = d_se.cpu().numpy()
    value = steps_done / (total_ms * 1e-3)
    se_c = np.sqrt((se ** 2).sum(-1))
    solves = int((se_c <= 1e-3).sum())

    # ---- end-to-end through the host-buffer C ABI (copies inside the timed region)
    e2e_steps, e2e_t, h2d, d2h = 0, 0.0, 0, 0
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, st = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], w["dt"], w["seed"] + k,
                                            node_ids=node_ids)
        e2e_t += time.perf_counter() - t0
        e2e_steps += st["steps"]
        h2d, d2h = st["h2d_bytes"], st["d2h_bytes"]
        kernel_ms_host = st["kernel_ms"]
    e2e_value = e2e_steps / e2e_t

    # ---- interface-node solves at standard error 1e-3 (adaptive path counts)
    solve_ms, met, walks_t = [], 0, 0
    for k in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, se_t, used, st_t = sdd.sdd_interface_values_target(
            ctx, w["nodes"], 4096, 4_000_000, 1e-3, w["dt"], w["seed"] + 100 + k, node_ids=node_ids)
        solve_ms.append(1e3 * (time.perf_counter() - t0))
        met = int((np.sqrt((se_t ** 2).sum(-1)).max(-1) <= 1e-3).sum())
        walks_t = int(used.sum())
    solve_s = statistics.mean(solve_ms) * 1e-3

    peaks, src = load_peaks()
    clk_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tinst = n_sm * 128 * clk_mhz * 1e6 / 1e12
    walk_ms = statistics.mean(step_ms)  # walk kernel dominates each step (ncu share in profiles/)
    achieved = INST_PER_STEP * steps_done_one / (walk_ms * 1e-3) / 1e12

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": (f"quarterspace: {n} nodes on x=0, z in [0,0.9], "
                                    f"{int(w['n_paths'][0])} walks/node, dt 1e-4, kappa 2|20 earth, "
                                    "0 air (dimensionless)"),
                       "walks_per_step": int(n * w["n_paths"][0]),
                       "steps_per_step": int(steps_done_one),
                       "l2": "flushed between steps (256 MB write)",
                       "precision": "FP32 walk, FP64 sums",
                       "launch": tuned if tuned else "default shape",
                       "cuda_graph": bool(args.graph)},
            "node_solves": {"value": met / solve_s, "unit": "interface-node solves/s",
                            "target_se": 1e-3, "nodes_met": f"{met}/{n}", "pilot": 4096,
                            "n_max": 4_000_000, "walks_per_solve_set": walks_t,
                            "ms_per_solve_set": 1e3 * solve_s,
                            "how": "sdd_interface_values_target, host buffers, pilot + top-up"},
            "fixed_count_nodes_at_se_1e-3": f"{solves}/{n}",
            "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tinst,
                         "unit": "Tinst/s", "frac": achieved / peak_tinst,
                         "traffic": None if args.small else traffic_per_launch(),
                         "peak_source": f"{n_sm} SMs x 128 lanes x {clk_mhz:.0f} MHz ({src} max clock)",
                         "inst_per_step": INST_PER_STEP},
            "clocks": clocks,
            "gpu_launches": 2 * args.steps,
        }
        objs = set(args.objects.split(",")) if args.objects != "all" else \
            {"serving", "tm", "interp", "mt", "rbffd", "block", "triangle"}
        full = world == 1 and not args.small
        cpu = not args.no_cpu_baseline
        if full and cpu:
            # the FP32 walk against the oracle on the same streams: four nodes
            # of the line under their own node ids, their first 20000 walks
            line["fp32_error"], _ = fp32_error(sdd, ctx, w, [9, 32, 50, 63], 20000, w["dt"], w["seed"])
        if full and "block" in objs:
            line["block"] = block_measure(sdd, torch, dev, peak_tinst, flush, cpu=cpu, tune=not args.no_autotune)
        if full and "triangle" in objs:
            line["triangle"] = triangle_measure(sdd, torch, dev, peak_tinst, flush, cpu=cpu,
                                                tune=not args.no_autotune)
        if args.small and world == 1 and args.objects != "all":
            # small cases of the block and triangle programs (for profiler
            # captures): 64 of the block's nodes with 1/8 of their walks; 16 of
            # the triangle's nodes x 1e5 walks at dt 1e-4; two launches each
            line["small_cases"] = small_cases(sdd, objs)
        if args.serve_requests > 0 and full and "serving" in objs:
            line["serving"] = serving(sdd, args.serve_requests)
        if full and "tm" in objs:
            line["tm"] = tm_measure(sdd, torch, dev, peak_tinst, max(1, min(args.steps, 3)), cpu=cpu,
                                    tune=not args.no_autotune)
        if full and "interp" in objs:
            line["interp"] = interp_measure(sdd, cpu=cpu)
        if full and "mt" in objs:
            line["mt"] = mt_measure(sdd, cpu=cpu)
        if full and "rbffd" in objs:
            line["rbffd"] = rbffd_measure(sdd, cpu=cpu)
        if cpu and world == 1:
            cb = cpu_baseline(w)
            cb.pop("seconds", None)
            line["cpu_baseline"] = cb
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())

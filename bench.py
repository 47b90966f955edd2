#!/usr/bin/env python
"""Benchmark: connections built per second (generate + sort + index) on GB300.

One step builds every network of the two-population rule sweep (2 x 100,000
nodes, four Connect calls of one rule; fixed_indegree / fixed_outdegree
K = 1,000, fixed_total_number 1e8 per call, pairwise_bernoulli p = 0.01,
all_to_all on 2 x 10,000, one_to_one on 2 x 100,000; each with multapses and
autapses allowed, and both forbidden), i.e. CreatePopulation -> Connect ->
Finalize -> GetConnections for 12 networks, about 4e9 connections.

Prints one JSON line.  `value` is device-timed (CUDA events on the stream the
library runs on); `e2e` is host wall-clock through the public API.  With
--impl reference the CPU oracle is timed instead, on a bounded sample.
Under torchrun each rank builds the same workload independently (replicas:
the construction path has no exchange step) and rank 0 reports the total.
"""
from __future__ import annotations

import argparse
import csv
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "connections built/sec (generate+sort+index) on 1 GB300, % HBM roofline; p50/p99 latency"
E2E_STEPS = 3  # timed end-to-end passes, after one untimed pass


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="snc", choices=["snc", "reference"])
    ap.add_argument("--workload", default="rule_sweep",
                    choices=["rule_sweep", "microcircuit", "plain", "small", "profile", "profile_total",
                             "profile_sampler", "profile_bernoulli", "profile_outdegree", "batched", "served",
                             "trials", "deliver", "profile_deliver"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="rule sweep only: skip the microcircuit, batched and served lines")
    ap.add_argument("--sort-digit-bits", type=int, default=None, help="tuning: widest radix digit")
    ap.add_argument("--sort-group-tiles", type=int, default=None, help="tuning: tiles per look-back unit")
    ap.add_argument("--sort-items", type=int, default=None, help="tuning: keys per thread of the bulk-copy pass")
    return ap.parse_args()


def workload_specs(name):
    from paper_2306_09855_gb300 import workloads as W
    if name == "rule_sweep":
        return [W.rule_sweep(r, m) for r, m in W.RULE_SWEEP_RUNS], {
            "workload": "rule sweep: 2 x 100,000 nodes, 4 Connect calls of one rule per network "
                        "(fixed_indegree/outdegree K=1000, fixed_total_number 1e8/call, "
                        "pairwise_bernoulli p=0.01, all_to_all 2 x 10,000, one_to_one 2 x 100,000), "
                        "multapses+autapses on and off: 12 networks",
            "seed": 1234, "dt_ms": 0.1}
    if name == "microcircuit":
        return [W.microcircuit()], {"workload": "microcircuit-shaped: 8 populations, 77,169 nodes, "
                                                "64 fixed_total_number calls, 3.0e8 connections",
                                    "seed": 1234, "dt_ms": 0.1}
    if name == "plain":
        return [W.plain_indegree()], {"workload": "2 x 1,000 nodes, fixed_indegree K=100, 400k connections",
                                      "seed": 1234, "dt_ms": 0.1}
    if name == "profile":
        return [W.two_population(100_000, "fixed_indegree", k=100)], {
            "workload": "profiling case: 2 x 100,000 nodes, fixed_indegree K=100 (4e7 connections, "
                        "same 43-bit key as the rule sweep)", "seed": 1234}
    if name == "batched":
        return W.batched_sweep(64), {
            "workload": "batched: 64 independent two-population networks, N per population log-uniform "
                        "2,000-50,000, fixed_indegree K 50-2,000 / fixed_total_number / pairwise_bernoulli "
                        "p 0.005-0.05, per-instance seeds, built by one snc_batch_finalize",
            "seed": 1234, "dt_ms": 0.1}
    if name == "profile_total":
        return [W.two_population(30_000, "fixed_total_number", k=20_000_000, autapses=False, multapses=False)], {
            "workload": "profiling case: 2 x 30,000 nodes, fixed_total_number 2e7 per call without autapses "
                        "or multapses (8e7 connections)", "seed": 1234}
    if name == "profile_sampler":
        return [W.two_population(100_000, "fixed_indegree", k=100, autapses=False, multapses=False)], {
            "workload": "profiling case: 2 x 100,000 nodes, fixed_indegree K=100 without autapses or "
                        "multapses (4e7 connections)", "seed": 1234}
    if name == "profile_outdegree":
        return [W.two_population(20_000, "fixed_outdegree", k=1000)], {
            "workload": "profiling case: 2 x 20,000 nodes, fixed_outdegree K=1000 (8e7 connections, sorted per "
                        "source by delay step)", "seed": 1234}
    if name == "profile_bernoulli":
        return [W.two_population(100_000, "pairwise_bernoulli", p=0.001, autapses=False)], {
            "workload": "profiling case: 2 x 100,000 nodes, pairwise_bernoulli p=0.001 (about 4e7 "
                        "connections)", "seed": 1234}
    return [W.rule_sweep("fixed_indegree", True, scale=0.1)], {
        "workload": "small: 2 x 10,000 nodes fixed_indegree K=1000", "seed": 1234}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def committed_traffic():
    """DRAM bytes per element of one radix pass from the committed ncu summary,
    or None when the sort kernels changed since those counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "onesweep_traffic.json")) as f:
            tr = json.load(f)
        with open(os.path.join(ROOT, "paper_2306_09855_gb300", "csrc", "sort_kernels.cu"), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != tr.get("sort_kernels_cu_sha1"):
                return None
        return tr
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sms, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as f:
                for row in csv.reader(f):
                    if len(row) < 9:
                        continue
                    try:
                        sms.append(float(row[1]))
                        maxes.append(float(row[2]))
                    except ValueError:
                        continue
                    for name, v in zip(names, row[5:9]):
                        if v.strip().lower() == "active":
                            reasons.add(name)
        finally:
            os.unlink(self.path)
        if not sms:
            return None
        sms.sort()
        return {"sm_mhz": sms[len(sms) // 2], "sm_max_mhz": max(maxes), "reasons": sorted(reasons),
                "samples": len(sms)}


def host_info():
    """nproc, CPU model and machine of the host the oracle runs on."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def cpu_baseline(sample_syn_target=1e7):
    """The oracle (as it stands) on a bounded sample of the workload, on one
    core and on every core (its OpenMP form, pinned equal to the
    single-thread oracle)."""
    import oracle
    from paper_2306_09855_gb300 import workloads as W
    spec = W.rule_sweep("fixed_indegree", True, scale=0.05)  # 2 x 5,000 nodes, K = 1,000: 2e7
    t0 = time.perf_counter()
    out = oracle.build(spec)
    dt = time.perf_counter() - t0
    n = out["src"].size
    del out
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    par = oracle.build_parallel(spec, threads)
    dt_par = time.perf_counter() - t0
    assert par["src"].size == n
    del par
    return {"value": n / dt, "unit": "connections/s", "cores": 1, "kind": "oracle",
            "sample": "fixed_indegree K=1000 on 2 x 5,000 nodes (%d connections), single-threaded C "
                      "oracle: generate + stable sort + index, %.1f s" % (n, dt),
            "omp": {"value": n / dt_par, "unit": "connections/s", "cores": threads, "seconds": dt_par,
                    "note": "the same oracle on every host thread (OpenMP: primary nodes and the merge sort "
                            "in parallel; pinned equal to the single-thread oracle)"},
            "host": host_info()}


def run_reference(args):
    """--impl reference: the CPU oracle timed on host cores, bounded samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2306_09855_gb300 import workloads as W
    spec = W.rule_sweep("fixed_indegree", True, scale=0.025)  # 2 x 2,500 nodes, K = 1,000: 1e7
    for _ in range(args.warmup):
        oracle.build(spec)
    t0 = time.perf_counter()
    n = 0
    for _ in range(args.steps):
        n += oracle.build(spec)["src"].size
    dt = time.perf_counter() - t0
    value = n / dt
    sample = "fixed_indegree K=1000 on 2 x 2,500 nodes (%d connections per step)" % (n // max(1, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "connections/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32+f32", "data": "synthetic",
            "config": workload_specs(args.workload)[1],
            "cpu_baseline": {"value": value, "unit": "connections/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "connections/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


def _serve(snc, srv, specs, arrivals, hold_s):
    """Submit specs at the given arrival offsets (seconds; None = all at
    once), collect every completion on a second thread, keep each network
    resident for hold_s seconds after it finished, then release it.
    Returns (wall seconds, per-request records, stats, host bytes)."""
    import collections
    import threading
    done = []
    io = {"h2d": 0, "d2h": 0}
    t0 = time.perf_counter()

    def completer():
        held = collections.deque()
        while len(done) < len(specs):
            t = srv.wait_any(timeout_ms=20)
            now = time.perf_counter()
            while held and (held[0][0] <= now or t == 0 and len(done) == len(specs)):
                srv.release(held.popleft()[1])
            if t == 0:
                continue
            v = srv.view(t)
            tm = srv.times(t)
            st = snc.snc_get_stats(snc.snc_server_context(srv.srv, t))
            io["h2d"] += int(st.h2d_bytes)
            io["d2h"] += int(st.d2h_bytes)
            done.append((int(v.n_syn), tm.latency_ms, tm.queued_ms, tm.batch_size, now))
            if hold_s > 0:
                held.append((now + hold_s, t))
            else:
                srv.release(t)
        while held:
            srv.release(held.popleft()[1])

    th = threading.Thread(target=completer)
    th.start()
    for i, sp in enumerate(specs):
        if arrivals is not None:
            wait = t0 + arrivals[i] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
        srv.submit(sp)
    th.join()
    last = max(r[4] for r in done)
    return last - t0, done, srv.stats(), io


def run_served(args, count=2000):
    """Served form: a Poisson stream of 2,000 construction requests (sizes
    log-uniform 1e5-5e8, rule uniform over the six, multapses on or off),
    admitted under a 150 GB budget, results resident until released.
    Returns the JSON line."""
    import torch
    from paper_2306_09855_gb300 import snc
    from paper_2306_09855_gb300 import workloads as W
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    snc.load()
    stream_specs = W.served_stream(count)
    specs = [sp for _, sp in stream_specs]
    offsets = [t for t, _ in stream_specs]
    budget = 150 * 10**9
    slots, batch_nets, batch_syn = 4, 64, 40_000_000

    def plain(spec_list):
        n = 0
        t0 = time.perf_counter()
        for sp in spec_list:
            net = snc.Network(sp, device=local)
            net.finalize()
            n += int(net.view().n_syn)
            net.close()
        torch.cuda.synchronize()
        return n, time.perf_counter() - t0

    for sp in specs[:max(3, args.warmup)]:
        plain([sp])
    # Plain-path capacity on the first 200 requests of the stream.
    n_cap, t_cap = plain(specs[:200])
    capacity = 200 / t_cap
    rate = 0.7 * capacity
    arrivals = [o / rate for o in offsets]
    torch.cuda.empty_cache()

    srv = snc.Server(budget, device=local, max_slots=slots, batch_max_nets=batch_nets, batch_max_syn=batch_syn)
    try:
        _serve(snc, srv, specs[:32], None, 0.0)  # warm the pool and the workers
        clocks = ClockSampler(local)
        clocks.start()
        torch.cuda.synchronize()
        wall, recs, st, io = _serve(snc, srv, specs, arrivals, hold_s=0.5)
        clk = clocks.stop()
        sat_wall, sat_recs, sat_st, _ = _serve(snc, srv, specs, None, 0.0)
    finally:
        srv.close()
    torch.cuda.empty_cache()
    n_plain, t_plain = plain(specs)
    n_total = sum(r[0] for r in recs)
    lat = [r[1] for r in recs]
    sat_lat = [r[1] for r in sat_recs]
    line = {
        "metric": METRIC, "value": n_total / wall, "unit": "connections/s", "n_gpus": 1,
        "steps": 1, "warmup": max(3, args.warmup), "ms_per_step": wall * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32+f32",
        "data": "synthetic",
        "config": {"workload": "served: %d two-population construction requests, Poisson arrivals, " % count +
                               "sizes log-uniform 1e5-5e8 connections, rule uniform over the six, "
                               "multapses on/off, 150 GB budget, networks held 0.5 s after completion",
                   "seed": 1234, "arrival_rate_per_s": rate, "plain_capacity_req_per_s": capacity,
                   "budget_bytes": budget, "max_slots": slots, "batch_max_nets": batch_nets,
                   "batch_max_syn": batch_syn, "connections": n_total,
                   "l2": "inputs larger than L2 for most of the work (requests above 1e7 connections)",
                   "timing": "host wall clock, submit of the first request to completion of the last"},
        "latency_ms": {"p50": _percentile(lat, 50), "p99": _percentile(lat, 99),
                       "mean": sum(lat) / len(lat), "max": max(lat)},
        "server": {"builds": int(st.builds), "batched_builds": int(st.batched_builds),
                   "peak_reserved_bytes": int(st.peak_reserved_bytes)},
        "saturated": {"value": sum(r[0] for r in sat_recs) / sat_wall, "unit": "connections/s",
                      "note": "all %d requests submitted at once, released on completion" % count,
                      "latency_ms": {"p50": _percentile(sat_lat, 50), "p99": _percentile(sat_lat, 99)},
                      "builds": int(sat_st.builds) - int(st.builds),
                      "batched_builds": int(sat_st.batched_builds) - int(st.batched_builds)},
        "plain_sequential": {"value": n_plain / t_plain, "unit": "connections/s",
                             "note": "the same %d requests built one after another with snc_finalize" % count},
        "roofline": None,
        "gpu_launches": None,
        "e2e": {"value": n_total / wall, "unit": "connections/s", "h2d_bytes_per_step": io["h2d"],
                "d2h_bytes_per_step": io["d2h"],
                "note": "the served stream through the public API; networks stay on the device"},
        "clocks": clk,
    }
    return line


def run_trials(args):
    """Repeated construction of the microcircuit-shaped network with new seeds
    (the paper's repeated trials, Sec. 2.7): each step rebuilds it by replaying
    the recorded CUDA graph of the build, against the plain path that
    finalizes a fresh context per seed."""
    import torch
    from dataclasses import replace
    from paper_2306_09855_gb300 import snc
    from paper_2306_09855_gb300 import workloads as W
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    snc.load()
    base = W.microcircuit()
    stream = torch.cuda.current_stream()
    steps, warm = args.steps, max(3, args.warmup)

    def timed(fn, n):
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        start.record(stream)
        total = 0
        for i in range(n):
            total += fn(i)
        end.record(stream)
        torch.cuda.synchronize()
        return total, start.elapsed_time(end), time.perf_counter() - t0

    def plain(i):
        net = snc.Network(replace(base, seed=5000 + i), stream=stream).finalize()
        n = int(net.view().n_syn)
        net.close()
        return n

    nets = snc.Network.batch_graph([base], stream=stream)

    def graph(i):
        nets[0].rebuild([5000 + i])
        return int(nets[0].view().n_syn)

    for i in range(warm):
        plain(i)
        graph(i)
    clocks = ClockSampler(local)
    clocks.start()
    n_g, ms_g, wall_g = timed(graph, steps)
    clk = clocks.stop()
    n_p, ms_p, wall_p = timed(plain, steps)
    nets[0].close()
    line = {
        "metric": METRIC, "value": n_g / (ms_g / 1e3), "unit": "connections/s", "n_gpus": 1, "steps": steps,
        "warmup": warm, "ms_per_step": ms_g / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32+f32", "data": "synthetic",
        "config": {"workload": "repeated trials: the microcircuit-shaped network (8 populations, 77,169 nodes, "
                               "64 fixed_total_number calls, 3.0e8 connections) rebuilt with a new seed per step by "
                               "replaying the recorded CUDA graph of its build", "seeds": "5000 + step",
                   "l2": "inputs larger than L2"},
        "plain_path": {"value": n_p / (ms_p / 1e3), "unit": "connections/s", "ms_per_build": ms_p / steps,
                       "note": "a fresh context finalized per seed (host planning, allocation, launches)"},
        "roofline": None,
        "gpu_launches": steps,
        "e2e": {"value": n_g / wall_g, "unit": "connections/s", "h2d_bytes_per_step": 8, "d2h_bytes_per_step": 64,
                "note": "host wall clock through snc_batch_rebuild; networks stay on the device"},
        "clocks": clk,
    }
    print(json.dumps(line))


def run_deliver(args):
    """Spike delivery through the index (Sec. 2.3), the step after
    construction: the rule sweep's fixed_indegree network (2 x 100,000 nodes,
    4e8 connections) receives per step a spike array of 10^6 entries (random
    source and connection group, multiplicity in [0.5, 2])."""
    import torch
    from paper_2306_09855_gb300 import snc
    from paper_2306_09855_gb300 import workloads as W
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    snc.load()
    small = args.workload == "profile_deliver"
    spec = W.two_population(100_000, "fixed_indegree", k=100) if small else W.rule_sweep("fixed_indegree", True)
    stream = torch.cuda.current_stream()
    net = snc.Network(spec, stream=stream).finalize()
    v = net.view()
    n_nodes = int(v.n_nodes)
    gp = torch.empty(n_nodes + 1, dtype=torch.int64, device="cuda")
    host = snc.snc_copy_index(net.ctx, n_nodes, int(v.n_groups))
    gp.copy_(torch.from_numpy(host["group_ptr"].view(np.int64)))
    n_spikes = 200_000 if small else 1_000_000
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1234)
    groups = (gp[1:] - gp[:-1])

    have = torch.nonzero(groups > 0).flatten()  # sources with connections

    def spike_array():
        src = have[torch.randint(0, have.numel(), (n_spikes,), device="cuda", generator=gen, dtype=torch.int64)]
        grp = (torch.rand(n_spikes, device="cuda", generator=gen) * groups[src]).to(torch.int64)
        grp = torch.minimum(grp, groups[src] - 1)
        mult = torch.rand(n_spikes, device="cuda", generator=gen) * 1.5 + 0.5
        return src.to(torch.int32), grp.to(torch.int32), mult.to(torch.float32).contiguous()

    arrays = [spike_array() for _ in range(4)]
    sizes = []
    row = torch.from_numpy(host["row_ptr"].view(np.int64)).cuda()
    gfirst = torch.from_numpy(host["group_first"].view(np.int64)).cuda()
    for src, grp, _ in arrays:  # connections each array delivers (for the metric)
        g = gp[src.long()] + grp.long()
        nxt = torch.where(grp.long() + 1 < groups[src.long()], gfirst[torch.clamp(g + 1, max=gfirst.numel() - 1)],
                          row[src.long() + 1])
        sizes.append(int((nxt - gfirst[g]).sum()))
    inp = torch.zeros(n_nodes, dtype=torch.float32, device="cuda")
    steps, warm = args.steps, max(3, args.warmup)
    for i in range(warm):
        s, g, m = arrays[i % 4]
        net.deliver(s, g, m, inp)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    n_conn = 0
    for i in range(steps):
        s, g, m = arrays[i % 4]
        net.deliver(s, g, m, inp)
        n_conn += sizes[i % 4]
    end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = start.elapsed_time(end)
    # Per delivered connection: target 4 B + weight 4 B read; the input is an
    # 800 KB array of L2-resident atomic adds.
    peak, peak_src = measured_peaks()
    achieved = 8.0 * n_conn / (ms / 1e3) / 1e9
    net.close()
    line = {
        "metric": "spike deliveries/sec (connections delivered through the index) on 1 GB300", "value": n_conn / (ms / 1e3),
        "unit": "connections/s", "n_gpus": 1, "steps": steps, "warmup": warm, "ms_per_step": ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": ("profiling case: fixed_indegree 2 x 100,000 nodes, K=100 (4e7 connections), "
                                "2e5 spike-array entries per step") if small else
                               ("spike delivery: rule-sweep fixed_indegree network (2 x 100,000 nodes, K=1000, 4e8 "
                                "connections), 10^6 spike-array entries per step (random source and group)"),
                   "connections_per_step": n_conn // max(1, steps), "l2": "target and weight arrays larger than L2"},
        "roofline": {"bound": "hbm", "kernel": "deliver_kernel", "achieved": achieved, "peak": peak,
                     "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "note": "8 B read per connection; the fp32 atomic adds go to an L2-resident input array"},
        "gpu_launches": 5 * steps,
        "e2e": {"value": n_conn / (ms / 1e3), "unit": "connections/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 8,
                "note": "the spike arrays and the input stay on the device; snc_deliver reads its error word back"},
        "clocks": clk,
    }
    print(json.dumps(line))


def _digest(torch, net):
    """Position-weighted sums of a built network's device arrays (equal
    networks give equal digests; int64 sums wrap deterministically)."""
    t = net.tensors()
    out = [int(t["target"].numel()), int(t["group_first"].numel())]
    for name in ("target", "delay", "weight", "row_ptr", "group_ptr", "group_first"):
        x = t[name]
        if x.numel() == 0:
            out.append(0)
            continue
        x = x.view(torch.int32) if x.dtype == torch.float32 else x
        x = x.to(torch.int64) & (0xFFFF if name == "delay" else -1)
        w = torch.arange(x.numel(), device=x.device, dtype=torch.int64) % 65521 + 1
        out.append(int((x * w).sum()))
    return tuple(out)


def _device_ms(torch, stream, fn):
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    r = fn()
    end.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(end), r


def extra_microcircuit(torch, snc, local, stream, steps=5, warm=3):
    """The microcircuit-shaped network (3.0e8 connections, 64
    fixed_total_number calls): device-timed builds, as the main line."""
    from paper_2306_09855_gb300 import workloads as W
    spec = W.microcircuit()

    def build():
        net = snc.Network(spec, device=local, stream=stream).finalize()
        n = int(net.view().n_syn)
        net.close()
        return n

    for _ in range(warm):
        build()
    ms, n = _device_ms(torch, stream, lambda: sum(build() for _ in range(steps)))
    return {"value": n / (ms / 1e3), "unit": "connections/s", "ms_per_build": ms / steps,
            "connections": n // steps, "steps": steps, "warmup": warm,
            "workload": "microcircuit-shaped: 8 populations, 77,169 nodes, 64 fixed_total_number calls"}


def extra_batched(torch, snc, local, stream, steps=3, warm=2):
    """64 networks of uneven size built by one snc_batch_finalize against the
    same 64 built one after another with snc_finalize (device time), with
    every member's arrays compared between the two (digests)."""
    from paper_2306_09855_gb300 import autotune
    from paper_2306_09855_gb300 import workloads as W
    specs = W.batched_sweep(64)
    saved = snc.snc_get_tuning()
    try:
        tune_info = autotune.tune(specs, batched=True)

        def batched():
            nets = snc.Network.batch(specs, device=local, stream=stream)
            n = sum(int(x.view().n_syn) for x in nets)
            return nets, n

        def sequential():
            nets = [snc.Network(sp, device=local, stream=stream).finalize() for sp in specs]
            n = sum(int(x.view().n_syn) for x in nets)
            return nets, n

        def timed(fn):
            for _ in range(warm):
                nets, _ = fn()
                for x in reversed(nets):
                    x.close()
            total_ms, total_n = 0.0, 0
            for _ in range(steps):
                ms, (nets, n) = _device_ms(torch, stream, fn)
                total_ms += ms
                total_n += n
                for x in reversed(nets):
                    x.close()
            return total_n / (total_ms / 1e3), total_ms / steps, total_n // steps

        v_b, ms_b, n_b = timed(batched)
        v_s, ms_s, n_s = timed(sequential)
        nets_b, _ = batched()
        dig_b = [_digest(torch, x) for x in nets_b]
        for x in reversed(nets_b):
            x.close()
        nets_s, _ = sequential()
        dig_s = [_digest(torch, x) for x in nets_s]
        for x in reversed(nets_s):
            x.close()
        # The same 64 as one recorded CUDA graph, rebuilt with new seeds per
        # step (Bernoulli totals and redraw rounds decided on the device),
        # then with the original seeds again (must equal the batched build).
        gnets = snc.Network.batch_graph(specs, device=local, stream=stream)
        try:
            def rebuild(step):
                def fn():
                    gnets[0].rebuild([sp.seed + 1000 * (step + 1) for sp in specs])
                    return sum(int(x.view().n_syn) for x in gnets)
                return fn
            for w in range(warm):
                rebuild(w)()
            g_ms, g_n = 0.0, 0
            for k in range(steps):
                ms, n = _device_ms(torch, stream, rebuild(warm + k))
                g_ms += ms
                g_n += n
            gnets[0].rebuild([sp.seed for sp in specs])
            dig_g = [_digest(torch, x) for x in gnets]
        finally:
            for x in reversed(gnets):
                x.close()
    finally:
        snc.snc_set_tuning(sort_digit_bits=saved.sort_digit_bits, sort_group_tiles=saved.sort_group_tiles,
                           gen_blocks_per_sm=saved.gen_blocks_per_sm, sort_items=saved.sort_items)
    return {"value": v_b, "unit": "connections/s", "ms_per_build": ms_b, "connections": n_b,
            "sequential_builds": {"value": v_s, "unit": "connections/s", "ms": ms_s, "connections": n_s},
            "speedup": v_b / v_s, "identical": dig_b == dig_s and n_b == n_s,
            "graph_rebuild": {"value": g_n / (g_ms / 1e3), "unit": "connections/s", "ms_per_build": g_ms / steps,
                              "identical_at_the_original_seeds": dig_g == dig_b,
                              "note": "the 64 networks recorded once as a CUDA graph (snc_batch_finalize_graph) "
                                      "and rebuilt with new seeds per step (snc_batch_rebuild); device time "
                                      "through the views' refresh"},
            "tuning": tune_info["tuning"], "tuning_cached": tune_info["cached"],
            "workload": "64 two-population networks, N log-uniform 2,000-50,000, fixed_indegree / "
                        "fixed_total_number / pairwise_bernoulli, per-instance seeds"}


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "served":
        print(json.dumps(run_served(args)))
        return
    if args.workload == "trials":
        run_trials(args)
        return
    if args.workload in ("deliver", "profile_deliver"):
        run_deliver(args)
        return
    import torch
    from paper_2306_09855_gb300 import replicas
    rank, world, local = replicas.world()
    torch.cuda.set_device(local)
    replicas.init("nccl")
    from paper_2306_09855_gb300 import snc
    snc.load()
    tuning = snc.snc_set_tuning(sort_digit_bits=args.sort_digit_bits, sort_group_tiles=args.sort_group_tiles,
                                sort_items=args.sort_items)
    specs, config = workload_specs(args.workload)
    stream = torch.cuda.current_stream()

    barrier = replicas.barrier

    batched = args.workload == "batched"
    tune_info = None
    if batched:
        from paper_2306_09855_gb300 import autotune
        tune_info = autotune.tune(specs, batched=True)

    def one_step(record):
        n_syn = 0
        if batched:
            nets = snc.Network.batch(specs, device=local, stream=stream)
            for net in nets:
                n_syn += int(net.view().n_syn)
            if record is not None:
                times, npass = nets[0].stage_times()
                record.append((n_syn, times, npass, nets[0].stats(), 0, 0))
            for net in reversed(nets):
                net.close()
            return n_syn
        for spec in specs:
            net = snc.Network(spec, device=local, stream=stream)
            net.finalize()
            v = net.view()  # synchronizes, reads the counts back
            n_syn += int(v.n_syn)
            if record is not None:
                times, npass = net.stage_times()
                st = net.stats()
                record.append((int(v.n_syn), times, npass, st, int(v.n_groups), int(v.n_nodes)))
            net.close()
        return n_syn

    for _ in range(max(3, args.warmup)):
        one_step(None)
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    records = []
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    start.record(stream)
    n_total = 0
    marks = []  # one event after each step (recorded in order; read after the final synchronize)
    for _ in range(args.steps):
        n_total += one_step(records)
        marks.append(torch.cuda.Event(enable_timing=True))
        marks[-1].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = start.elapsed_time(end)
    step_ms = [start.elapsed_time(marks[0])] + [marks[k - 1].elapsed_time(marks[k]) for k in range(1, len(marks))]
    ms, n_all = replicas.reduce_timing(ms, n_total, device="cuda")
    value = n_all / (ms / 1e3)

    # Dominant kernel: the onesweep radix pass.  Algorithmic bytes per launch:
    # read and write the key ((source, delay): 4 B, or 8 B above 32 bits)
    # and the value ((target, weight): 8 B): 24 B (32 B) per connection; the
    # last pass of a sort also writes the 2-byte delay array (it unpacks the
    # value into the target and weight arrays).
    pass_bytes, pass_ms, pass_launches = 0.0, 0.0, 0
    gen_bytes, gen_ms, launches = 0.0, 0.0, 0
    # Whole step: the bytes the method must move (generation writes the key
    # and value; each radix pass reads and writes them, the last one writing
    # the 2-byte delay array besides; the per-source sort reads them and
    # writes key, target, weight and delay; the index reads the sorted keys
    # once and writes the per-node and per-group offsets).
    step_bytes = 0.0
    stage_sum = {}
    for n_syn, times, npass, st, n_groups, n_nodes in records:
        launches += int(st.kernel_launches)
        key_b = 4.0 if st.key_bits <= 32 else 8.0
        pair = key_b + 8.0
        if st.source_major:
            # One per-source counting sort by delay instead of radix passes
            # (every projection generated source by source): not a radix pass.
            names = ["count", "generate", "source_offsets", "source_sort", "index"]
            step_bytes += (2.0 * pair + 2.0) * n_syn
        else:
            for k in range(npass):
                pass_bytes += (2.0 * pair + (2.0 if k == npass - 1 else 0.0)) * n_syn
                pass_ms += times[3 + k]
                pass_launches += 1
            names = ["count", "generate", "histogram"] + ["pass%d" % k for k in range(npass)] + ["index"]
            step_bytes += (2.0 * pair * npass + 2.0) * n_syn
        step_bytes += pair * n_syn + key_b * n_syn + 8.0 * n_groups + 16.0 * (n_nodes + 1)
        gen_bytes += pair * n_syn
        gen_ms += times[1]
        for nm, t in zip(names, times):
            stage_sum[nm] = stage_sum.get(nm, 0.0) + t
    per_network = None
    if not batched and records:
        per = {}
        for k, (n_syn, times, npass, st, _, _) in enumerate(records):
            name = specs[k % len(specs)].name
            e = per.setdefault(name, {"network": name, "connections": n_syn, "key_bits": int(st.key_bits),
                                      "passes": int(st.n_passes),
                                      "sort": "source-major" if st.source_major else "radix",
                                      "generate_ms": 0.0, "sort_ms": 0.0, "index_ms": 0.0})
            e["generate_ms"] += (times[0] + times[1]) / args.steps
            e["sort_ms"] += sum(times[2:3 + npass]) / args.steps
            e["index_ms"] += times[3 + npass] / args.steps
        per_network = list(per.values())
    final_tuning = snc.snc_get_tuning()
    peak, peak_src = measured_peaks()
    achieved = (pass_bytes / (pass_ms / 1e3)) / 1e9 if pass_ms > 0 else 0.0
    traffic = None
    tr = committed_traffic()
    if tr and pass_launches:
        # Keys moved by radix passes only (a source-major record's sort is not one).
        traffic = tr["dram_bytes_per_element"] * (sum(r[0] * r[2] for r in records if not r[3].source_major)) / pass_launches

    # End to end through the public API with host buffers: every step
    # plans on the host, copies the plans in, builds, and copies the whole
    # network as the device holds it (target, delay, weight: 10 B per
    # connection, plus row_ptr, p_i and group_first) back into page-locked
    # host arrays, all inside the host wall-clock region.  One host thread
    # queues network k's build on one of two streams and then copies network
    # k - 1 (built on the other stream) to the host, so that each copy
    # overlaps the next build and the copies follow one another on the link.
    max_syn = max(r[0] for r in records) if records else 0
    max_groups = max(max(r[4] for r in records), max_syn if batched else 0) if records else 0
    max_nodes = max(sp.n_nodes for sp in specs)

    def host_arrays():
        h = {name: torch.empty(max(1, size), dtype=dt, pin_memory=True).numpy()
             for name, dt, size in (("src", torch.int32, max_syn if batched else 1), ("tgt", torch.int32, max_syn),
                                    ("delay", torch.int16, max_syn), ("weight", torch.float32, max_syn),
                                    ("row_ptr", torch.int64, max_nodes + 1), ("group_ptr", torch.int64, max_nodes + 1),
                                    ("group_first", torch.int64, max_groups))}
        return {"src": h["src"].view(np.uint32), "tgt": h["tgt"].view(np.uint32),
                "delay": h["delay"].view(np.uint16), "weight": h["weight"],
                "row_ptr": h["row_ptr"].view(np.uint64), "group_ptr": h["group_ptr"].view(np.uint64),
                "group_first": h["group_first"].view(np.uint64)}

    host = host_arrays()
    streams = [torch.cuda.Stream(device=local) for _ in range(2)]
    # The builds above left their device blocks in torch's cache, tied to
    # their stream: hand them back so that the two streams below allocate
    # their own (otherwise a full cache is emptied mid-leg, and every free
    # waits for the whole device).
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    def e2e_pass():
        """One end-to-end pass over every network: (connections, h2d, d2h)."""
        if batched:
            n_p = d2h_p = 0
            nets = snc.Network.batch(specs, device=local, stream=stream)
            for net in nets:
                n_p += int(net.view().n_syn)
                net.to_host_network(host)
                d2h_p += int(net.stats().d2h_bytes)
            h2d_p = int(nets[0].stats().h2d_bytes)
            for net in reversed(nets):
                net.close()
            return n_p, h2d_p, d2h_p
        tot = [0, 0, 0]

        def drain(net):
            tot[0] += net.to_host_network(host)
            st = net.stats()
            tot[1] += int(st.h2d_bytes)
            tot[2] += int(st.d2h_bytes)
            net.close()

        prev = None
        for k, spec in enumerate(specs):
            net = snc.Network(spec, device=local, stream=streams[k % 2])
            net.finalize()  # queued (a Bernoulli count or a redraw round waits for its own stream)
            if prev is not None:
                drain(prev)
            prev = net
        if prev is not None:
            drain(prev)
        return tuple(tot)

    # One untimed pass warms the streams' allocations and the pinned
    # host pages; then E2E_STEPS timed passes (the bytes reported per pass).
    e2e_pass()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_e2e = 0
    e2e_pass_ms = []
    for _ in range(E2E_STEPS):
        tp = time.perf_counter()
        n_p, h2d, d2h = e2e_pass()
        e2e_pass_ms.append((time.perf_counter() - tp) * 1e3)
        n_e2e += n_p
    e2e_s = (time.perf_counter() - t0) / E2E_STEPS
    n_e2e //= E2E_STEPS
    e2e_ms_all, n_e2e_all = replicas.reduce_timing(e2e_s * 1e3, n_e2e, device="cuda")
    sequential = None
    if batched:
        from paper_2306_09855_gb300 import autotune
        seq_ms = autotune.time_build(specs, batched=False, repeats=1)
        sequential = {"value": n_e2e / (seq_ms / 1e3), "unit": "connections/s", "ms": seq_ms,
                      "note": "the same 64 networks built one after another with snc_finalize"}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "connections/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "step_ms": {"median": sorted(step_ms)[len(step_ms) // 2], "min": min(step_ms), "max": max(step_ms)},
        "dtype": "u32+f32", "data": "synthetic",
        "config": dict(config, connections_per_step=n_total // max(1, args.steps),
                       tuning={"sort_digit_bits": final_tuning.sort_digit_bits,
                               "sort_group_tiles": final_tuning.sort_group_tiles,
                               "gen_blocks_per_sm": final_tuning.gen_blocks_per_sm,
                               "sort_items": final_tuning.sort_items},
                       l2="inputs larger than L2 (>= 4.8 GB of keys+values per network)",
                       parallelism="replicas" if world > 1 else "single GPU"),
        "roofline": {"bound": "hbm", "kernel": "onesweep radix pass", "achieved": achieved, "peak": peak,
                     "peak_source": peak_src + " MEASURED_PEAKS.json hbm_gbs" if peak_src == "measured" else peak_src,
                     "unit": "GB/s", "frac": achieved / peak if peak else None, "traffic": traffic,
                     "launches": pass_launches, "avg_launch_ms": pass_ms / max(1, pass_launches),
                     "algorithmic_bytes_per_launch": pass_bytes / max(1, pass_launches)},
        "step_roofline": {"bound": "hbm", "algorithmic_bytes_per_step": step_bytes / args.steps,
                          "achieved": (step_bytes / args.steps) / (ms / args.steps / 1e3) / 1e9, "peak": peak,
                          "unit": "GB/s",
                          "frac": ((step_bytes / args.steps) / (ms / args.steps / 1e3) / 1e9) / peak if peak else None,
                          "note": "whole step: generation, sort and index bytes the method must move (12 B "
                                  "written per connection, 24 B per radix pass plus the 2-byte delay array, "
                                  "the index's read of the sorted keys, per-node and per-group offsets), over "
                                  "the step's CUDA-event time"},
        "stage_ms_per_step": {k: v / args.steps for k, v in stage_sum.items()},
        "generate_GBps": (gen_bytes / (gen_ms / 1e3)) / 1e9 if gen_ms else None,
        "gpu_launches": launches,
        "e2e": {"value": n_e2e_all / (e2e_ms_all / 1e3), "unit": "connections/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "steps": E2E_STEPS, "warmup": 1, "pass_ms": [round(x, 1) for x in e2e_pass_ms],
                "note": "public API, host wall clock: plan, build, and copy of each network as held on the "
                        "device (target, delay, weight: 10 B per connection; row_ptr, p_i, group_first) into "
                        "page-locked host arrays; one host thread, two streams: network k is built while "
                        "network k - 1 is copied; mean of the timed passes after one untimed pass"},
        "clocks": clk,
    }
    if per_network:
        line["per_network"] = per_network
    if batched:
        line["sequential_builds"] = sequential
        line["autotune"] = {"tuning": tune_info["tuning"], "cached": tune_info["cached"], "key": tune_info["key"]}
    if args.workload == "rule_sweep" and world == 1 and not args.no_extras:
        # The paper's other model, the batched form and the served form on
        # the same GPU, beside the rule sweep (each reported on its own).
        for key, fn in (("microcircuit", lambda: extra_microcircuit(torch, snc, local, stream)),
                        ("batched", lambda: extra_batched(torch, snc, local, stream)),
                        ("served", lambda: run_served(args))):
            try:
                line[key] = fn()
            except Exception as exc:  # reported in the line, the rule sweep stands
                line[key] = {"error": "%s: %s" % (type(exc).__name__, exc)}
            torch.cuda.empty_cache()
        sv = line.get("served")
        if isinstance(sv, dict) and "latency_ms" in sv:
            line["served"] = {k: sv[k] for k in ("value", "unit", "latency_ms", "saturated", "plain_sequential",
                                                 "server", "config", "clocks") if k in sv}
            line["latency_ms"] = sv["latency_ms"]
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))


if __name__ == "__main__":
    main()

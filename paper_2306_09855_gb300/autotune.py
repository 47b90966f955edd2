"""Autotuner for the kernel parameters exposed by snc_set_tuning.

The parameters change speed only, never results (every variant is tested to
give identical networks).  For a workload class the tuner times each
candidate on a representative build, keeps the fastest, and caches the choice
per (GPU name, key-width class, size class) in a JSON file.
"""
from __future__ import annotations

import json
import os
import time
from typing import Dict, List, Sequence

from . import snc

# (sort digit bits, tiles per look-back unit, generation blocks per SM,
#  keys per thread of the bulk-copy pass)
CANDIDATES = [(9, 0, 8, 32), (9, 0, 8, 24), (9, 0, 8, 16), (8, 0, 8, 32), (8, 0, 8, 16), (8, 0, 8, 12),
              (9, 0, 4, 32), (9, 0, 16, 32), (11, 8, 8, 16)]
FIELDS = ("sort_digit_bits", "sort_group_tiles", "gen_blocks_per_sm", "sort_items")


def _apply(tuning):
    snc.snc_set_tuning(**dict(zip(FIELDS, tuning)))

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "snc_tuning.json")


def _size_class(n_connections: int) -> str:
    for limit, name in ((1e6, "tiny"), (3e7, "small"), (3e8, "medium")):
        if n_connections < limit:
            return name
    return "large"


def _connections(specs) -> int:
    """Expected number of connections of the specifications (Sec. 2.1 counts;
    pairwise_bernoulli its mean), for the size class of the cache key."""
    n = 0.0
    for sp in specs:
        for pj in sp.projections:
            ns, nt = int(pj.src[1]), int(pj.tgt[1])
            n += {"one_to_one": ns, "all_to_all": ns * nt, "fixed_indegree": int(pj.k) * nt,
                  "fixed_outdegree": int(pj.k) * ns, "fixed_total_number": int(pj.k),
                  "pairwise_bernoulli": float(pj.p) * ns * nt}[pj.rule]
    return int(n)


def _key_class(specs) -> str:
    nodes = sum(sp.n_nodes for sp in specs)
    return "src%d" % max(1, int(nodes - 1).bit_length())


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(0).replace(" ", "_")


def time_build(specs: Sequence, batched: bool, repeats: int = 2) -> float:
    """Best device time (ms) of building `specs` (batched or one by one)."""
    import torch
    best = float("inf")
    for _ in range(repeats + 1):
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record()
        if batched:
            nets = snc.Network.batch(specs)
            for net in nets:
                net.view()
        else:
            nets = []
            for sp in specs:
                net = snc.Network(sp).finalize()
                net.view()
                nets.append(net)
        end.record()
        torch.cuda.synchronize()
        for net in reversed(nets):
            net.close()
        best = min(best, start.elapsed_time(end))
    return best


def tune(specs: Sequence, batched: bool = True, candidates=CANDIDATES, cache_path: str = DEFAULT_CACHE,
         use_cache: bool = True) -> Dict:
    """Pick and apply the fastest candidate for this workload class."""
    key = "v4/%s/%s/%s/%s" % (_gpu_name(), _key_class(specs), _size_class(_connections(specs)),
                              "batch" if batched else "single")
    cache = {}
    if use_cache and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache and len(cache[key].get("tuning", ())) == len(FIELDS):
        choice = cache[key]
        _apply(choice["tuning"])
        return dict(choice, key=key, cached=True)
    results: List[Dict] = []
    for cand in candidates:
        _apply(cand)
        t0 = time.perf_counter()
        ms = time_build(specs, batched)
        results.append({"tuning": list(cand), "ms": ms, "tune_s": time.perf_counter() - t0})
    best = min(results, key=lambda r: r["ms"])
    _apply(best["tuning"])
    choice = {"tuning": best["tuning"], "ms": best["ms"], "all": results}
    if use_cache:
        cache[key] = choice
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return dict(choice, key=key, cached=False)

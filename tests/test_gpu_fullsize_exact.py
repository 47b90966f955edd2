"""Element-by-element parity at full size: every network the benchmark
builds (the rule sweep's twelve networks of about 4e8 connections each on
2 x 100,000 nodes, 2 x 10,000 for all_to_all; the microcircuit shape's 3.0e8
connections in 64 fixed_total_number calls) against the oracle's whole
network, built on the host's cores by the oracle's threaded form (pinned
equal to the single-thread oracle in test_oracle_parallel.py).  Every
source, target, delay step, row and group offset bit-exact; weights within
4 fp32 ulp.

Each case holds about 2 x 5.6 GB of host arrays plus the oracle's sort
buffers (2 x 24 B per connection); a host with too little memory skips."""
import os

import numpy as np
import pytest

from gpu_helpers import WEIGHT_ULP, ulp_diff
from paper_2306_09855_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [("microcircuit", True)] + list(W.RULE_SWEEP_RUNS)


def _host_bytes_free():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


@pytest.fixture(scope="module")
def snc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09855_gb300 import snc as mod
    mod.load()
    return mod


@pytest.mark.parametrize("rule,mult", CASES, ids=["%s-%s" % (r, "mult" if m else "nomult") for r, m in CASES])
def test_full_size_network_equals_oracle(snc, oracle_mod, rule, mult):
    spec = W.microcircuit() if rule == "microcircuit" else W.rule_sweep(rule, mult)
    n_est = 4.0e8
    free = _host_bytes_free()
    if free is not None and free < n_est * 80:
        pytest.skip("host memory: %.0f GB available, about %.0f GB needed" % (free / 1e9, n_est * 80 / 1e9))
    net = snc.Network(spec).finalize()
    try:
        got = net.to_host()
    finally:
        net.close()
    ref = oracle_mod.build_parallel(spec)
    _assert_equal_chunked(got, ref, spec.name)


def _assert_equal_chunked(got, ref, what, chunk=1 << 26):
    """assert_network_equal of gpu_helpers, in slices (no 8-byte copies of
    whole 4e8-element arrays)."""
    n = ref["src"].size
    assert got["src"].size == n, (what, got["src"].size, n)
    for f in ("row_ptr", "group_ptr"):
        np.testing.assert_array_equal(got[f], ref[f], err_msg=f"{what}:{f}")
    assert got["n_groups"] == ref["n_groups"], what
    np.testing.assert_array_equal(got["group_first"][:ref["n_groups"]], ref["group_first"], err_msg=what)
    worst = 0
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        for f in ("src", "tgt", "delay"):
            a, b = got[f][lo:hi], ref[f][lo:hi]
            if not np.array_equal(a, b):
                bad = lo + int(np.flatnonzero(a != b)[0])
                raise AssertionError(f"{what}:{f} differs first at {bad}: {got[f][bad]} vs {ref[f][bad]}")
        worst = max(worst, int(ulp_diff(got["weight"][lo:hi], ref["weight"][lo:hi]).max(initial=0)))
    assert worst <= WEIGHT_ULP, (what, worst)

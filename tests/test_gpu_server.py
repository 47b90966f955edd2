"""Served form (include/snc_server.h): requests built concurrently, in
batches and under a memory budget give exactly the networks they give alone,
and the budget holds requests back until memory is released."""
import time

import numpy as np
import pytest

from gpu_helpers import assert_network_equal
from paper_2306_09855_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("src", "tgt", "delay", "weight", "row_ptr", "group_ptr", "group_first")


@pytest.fixture(scope="module")
def snc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09855_gb300 import snc as mod
    mod.load()
    return mod


def _alone(snc, spec):
    net = snc.Network(spec).finalize()
    out = net.to_host()
    net.close()
    return out


def _mixed_requests():
    """Small requests of every rule, both multapse settings, sizes 1e4-3e6."""
    rng = np.random.default_rng(77)
    out = []
    for i in range(30):
        rule = W.RULES[i % 6]
        size = float(np.exp(rng.uniform(np.log(1e4), np.log(3e6))))
        out.append(W.served_request(size, rule, bool(i % 4 < 2), 5000 + i))
    return out


def test_results_alone_equal_results_in_the_mix(snc, oracle_mod):
    specs = _mixed_requests()
    srv = snc.Server(hbm_budget_bytes=40 << 30, max_slots=3, batch_max_nets=8, batch_max_syn=8_000_000)
    try:
        tickets = [srv.submit(sp) for sp in specs]
        seen = set()
        while len(seen) < len(tickets):
            t = srv.wait_any(timeout_ms=120_000)
            assert t != 0, "server stalled"
            seen.add(t)
        assert seen == set(tickets)
        st = srv.stats()
        assert st.completed == len(specs) and st.failed == 0
        assert st.batched_builds >= 1  # small neighbours were built together
        oracle_checked = 0
        for i, (sp, t) in enumerate(zip(specs, tickets)):
            assert srv.state(t) == snc.SNC_JOB_DONE
            got = srv.to_host(t)
            ref = _alone(snc, sp)
            for f in FIELDS:
                np.testing.assert_array_equal(got[f], ref[f], err_msg=f"request {i} {f}")
            assert got["n_groups"] == ref["n_groups"]
            tm = srv.times(t)
            assert tm.latency_ms >= tm.build_ms >= 0 and tm.batch_size >= 1
            if got["src"].size <= 400_000 and oracle_checked < 6:
                assert_network_equal(got, oracle_mod.build(sp), f"request {i}")
                oracle_checked += 1
        assert oracle_checked >= 3
        for t in tickets:
            srv.release(t)
        st = srv.stats()
        assert st.released == len(specs) and st.resident_bytes == 0 and st.reserved_bytes == 0
    finally:
        srv.close()


def test_budget_holds_a_request_until_memory_is_released(snc):
    a = W.two_population(2000, "fixed_indegree", k=200, seed=1)
    b = W.two_population(2000, "fixed_indegree", k=200, seed=2)
    ctx = snc.create_context(a)
    peak, resident, n = snc.snc_estimate_build(ctx)
    snc.snc_destroy(ctx)
    assert n == 4 * 2000 * 200 and resident < peak
    srv = snc.Server(hbm_budget_bytes=peak, max_slots=2, batch_max_nets=1)
    try:
        ta = srv.submit(a)
        tb = srv.submit(b)
        assert srv.wait_any(timeout_ms=60_000) == ta
        # a stays resident, so b (whose peak alone fills the budget) waits
        time.sleep(0.3)
        assert srv.state(tb) == snc.SNC_JOB_QUEUED
        assert srv.wait_any(timeout_ms=0) == 0
        srv.release(ta)
        assert srv.wait_any(timeout_ms=60_000) == tb
        assert srv.times(tb).queued_ms >= 300.0
        np.testing.assert_array_equal(srv.to_host(tb)["tgt"], _alone(snc, b)["tgt"])
        srv.release(tb)
    finally:
        srv.close()


def test_request_above_the_budget_is_refused(snc):
    srv = snc.Server(hbm_budget_bytes=1 << 20, max_slots=1)
    try:
        with pytest.raises(snc.SncError) as e:
            srv.submit(W.plain_indegree())
        assert e.value.name == "INVALID_ARG"
        assert srv.stats().submitted == 0
    finally:
        srv.close()


def test_server_state_errors(snc):
    srv = snc.Server(hbm_budget_bytes=8 << 30, max_slots=1)
    try:
        net = snc.Network(W.plain_indegree()).finalize()
        with pytest.raises(snc.SncError) as e:
            snc.snc_server_submit(srv.srv, net.ctx)
        assert e.value.name == "STATE"
        net.close()
        with pytest.raises(snc.SncError) as e:
            srv.release(12345)
        assert e.value.name == "INVALID_ARG"
    finally:
        srv.close()


def test_destroy_with_work_queued_and_resident(snc):
    srv = snc.Server(hbm_budget_bytes=16 << 30, max_slots=2, batch_max_nets=4)
    for s in range(6):
        srv.submit(W.two_population(1500, "pairwise_bernoulli", p=0.02, seed=s))
    assert srv.wait_any(timeout_ms=60_000) != 0
    srv.close()  # waits for the builds in progress and frees everything


@pytest.mark.parametrize("spec", [
    W.two_population(3000, "fixed_indegree", k=300, autapses=False, multapses=False, seed=3),
    W.two_population(3000, "pairwise_bernoulli", p=0.03, autapses=False, seed=4),
    W.two_population(1000, "fixed_total_number", k=400_000, autapses=False, multapses=False, seed=5),
    W.two_population(1500, "all_to_all", seed=6),
    W.microcircuit(scale=0.05),
], ids=["indegree_nomult", "bernoulli", "total_nomult", "all_to_all", "microcircuit"])
def test_estimate_bounds_the_build(snc, spec):
    net = snc.Network(spec, allocator=None)
    peak, resident, n_est = snc.snc_estimate_build(net.ctx)
    net.finalize()
    v = net.view()
    st = net.stats()
    assert v.n_syn <= n_est
    assert st.device_bytes_peak <= peak
    net.close()


def test_target_shards_are_served_alone(snc):
    """Target shards of one network, submitted together with small requests
    that could be batched: every shard is built alone and equals the shard
    built without the server."""
    spec = W.two_population(1200, "fixed_indegree", k=30, seed=41)
    bounds = [(0, 800), (800, 900), (1700, 700)]
    srv = snc.Server(hbm_budget_bytes=16 << 30, max_slots=2, batch_max_nets=8, batch_max_syn=8_000_000)
    try:
        tickets = []
        for first, n in bounds:
            net = snc.Network(spec, allocator=None, target_shard=(first, n))
            tickets.append(snc.snc_server_submit(srv.srv, net.ctx))
            net.ctx = None  # the server owns the context now
        small = [srv.submit(W.two_population(300, "fixed_indegree", k=20, seed=50 + i)) for i in range(3)]
        seen = set()
        while len(seen) < len(tickets) + len(small):
            t = srv.wait_any(timeout_ms=120_000)
            assert t != 0, "server stalled"
            seen.add(t)
        for (first, n), t in zip(bounds, tickets):
            assert srv.state(t) == snc.SNC_JOB_DONE
            assert srv.times(t).batch_size == 1
            alone = snc.Network(spec, target_shard=(first, n)).finalize()
            ref = alone.to_host()
            alone.close()
            got = srv.to_host(t)
            for f in FIELDS:
                np.testing.assert_array_equal(got[f], ref[f], err_msg=f"shard {first}: {f}")
        for t in tickets + small:
            srv.release(t)
    finally:
        srv.close()

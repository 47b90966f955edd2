"""Batched calibration (snc_batch_finalize): every member of a batch gets
exactly the network a single build gives it, and the oracle's network."""
import numpy as np
import pytest

from gpu_helpers import assert_network_equal
from paper_2306_09855_gb300 import workloads as W
from paper_2306_09855_gb300.workloads import Dist, NetworkSpec, Projection

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09855_gb300 import snc as mod
    mod.load()
    return mod


def _mixed_specs():
    specs = [
        W.two_population(700, "fixed_indegree", k=31, autapses=False, seed=1),
        W.two_population(333, "pairwise_bernoulli", p=0.05, autapses=False, seed=2),
        W.two_population(500, "fixed_total_number", k=40_000, autapses=False, multapses=False, seed=3),
        W.two_population(64, "fixed_indegree", k=40, autapses=False, multapses=False, seed=4),
        W.two_population(90, "all_to_all", autapses=False, seed=5),
        NetworkSpec(seed=6, dt=0.1, populations=[7], projections=[]),
        W.two_population(1200, "fixed_outdegree", k=17, seed=7),
        W.two_population(40, "one_to_one", autapses=False, seed=8),
    ]
    specs += W.batched_sweep(count=6, scale=0.05)
    return specs


def test_batch_members_equal_single_builds_and_oracle(snc, oracle_mod):
    specs = _mixed_specs()
    nets = snc.Network.batch(specs)
    for i, (spec, net) in enumerate(zip(specs, nets)):
        got = net.to_host()
        single = snc.Network(spec).finalize()
        alone = single.to_host()
        single.close()
        for f in ("src", "tgt", "delay", "weight", "row_ptr", "group_ptr", "group_first"):
            np.testing.assert_array_equal(got[f], alone[f], err_msg=f"member {i} {f}")
        assert got["n_groups"] == alone["n_groups"]
        assert_network_equal(got, oracle_mod.build(spec), f"member {i}")


def test_batch_views_outlive_the_first_member(snc, oracle_mod):
    specs = [W.two_population(300, "fixed_indegree", k=20, seed=s) for s in (10, 11, 12)]
    nets = snc.Network.batch(specs)
    nets[0].close()
    for spec, net in zip(specs[1:], nets[1:]):
        assert_network_equal(net.to_host(), oracle_mod.build(spec), "after leader closed")


def test_batch_argument_errors(snc):
    a = snc.Network(W.two_population(50, "fixed_indegree", k=5))
    with pytest.raises(snc.SncError) as e:
        snc.snc_batch_finalize([a.ctx, a.ctx])
    assert e.value.name == "INVALID_ARG"
    a.finalize()
    b = snc.Network(W.two_population(50, "fixed_indegree", k=5))
    with pytest.raises(snc.SncError) as e:
        snc.snc_batch_finalize([b.ctx, a.ctx])
    assert e.value.name == "STATE"


def _fixed_count_specs():
    from dataclasses import replace
    specs = [
        W.two_population(600, "fixed_indegree", k=40, autapses=False, multapses=False, seed=31),
        W.two_population(500, "fixed_outdegree", k=25, seed=32),
        W.two_population(400, "fixed_total_number", k=30_000, seed=33),
        W.two_population(120, "all_to_all", autapses=False, seed=34),
        W.two_population(300, "one_to_one", seed=35),
        W.microcircuit(scale=0.03, seed=36),
    ]
    return specs, replace


def test_graph_rebuild_equals_plain_builds_with_new_seeds(snc, oracle_mod):
    specs, replace = _fixed_count_specs()
    nets = snc.Network.batch_graph(specs)
    fields = ("src", "tgt", "delay", "weight", "row_ptr", "group_ptr", "group_first")
    first = [net.to_host() for net in nets]
    for i, (spec, got) in enumerate(zip(specs, first)):
        single = snc.Network(spec).finalize()
        alone = single.to_host()
        single.close()
        for f in fields:
            np.testing.assert_array_equal(got[f], alone[f], err_msg=f"first build {i} {f}")
    for trial, offset in enumerate((1000, 2000)):
        seeds = [sp.seed + offset + i for i, sp in enumerate(specs)]
        nets[2].rebuild(seeds)  # any member replays the whole build
        for i, (spec, net) in enumerate(zip(specs, nets)):
            got = net.to_host()
            ref_spec = replace(spec, seed=seeds[i])
            single = snc.Network(ref_spec).finalize()
            alone = single.to_host()
            single.close()
            for f in fields:
                np.testing.assert_array_equal(got[f], alone[f], err_msg=f"trial {trial} member {i} {f}")
            assert got["n_groups"] == alone["n_groups"]
            if i == 0:
                assert_network_equal(got, oracle_mod.build(ref_spec), f"trial {trial} vs oracle")
    # back to the original seeds: the first result again
    nets[0].rebuild([sp.seed for sp in specs])
    for i, net in enumerate(nets):
        got = net.to_host()
        for f in fields:
            np.testing.assert_array_equal(got[f], first[i][f], err_msg=f"replay {i} {f}")
    for net in reversed(nets):
        net.close()


def _graph_trials(snc, oracle_mod, specs, offsets, oracle_members):
    """Graph build of `specs`, then rebuilds with shifted seeds: every member
    equals its single build with those seeds (and the oracle for the members
    listed), and the original seeds give the first result back."""
    from dataclasses import replace
    fields = ("src", "tgt", "delay", "weight", "row_ptr", "group_ptr", "group_first")
    nets = snc.Network.batch_graph(specs)
    try:
        first = [net.to_host() for net in nets]
        for trial, offset in enumerate((0,) + tuple(offsets)):
            seeds = [sp.seed + offset + i * (offset > 0) for i, sp in enumerate(specs)]
            if offset:
                nets[-1].rebuild(seeds)
            for i, (spec, net) in enumerate(zip(specs, nets)):
                got = net.to_host()
                ref_spec = replace(spec, seed=seeds[i])
                single = snc.Network(ref_spec).finalize()
                alone = single.to_host()
                single.close()
                assert int(net.view().n_syn) == alone["tgt"].size, (trial, i)
                for f in fields:
                    np.testing.assert_array_equal(got[f], alone[f], err_msg=f"trial {trial} member {i} {f}")
                assert got["n_groups"] == alone["n_groups"]
                if i in oracle_members:
                    assert_network_equal(got, oracle_mod.build(ref_spec), f"trial {trial} member {i} vs oracle")
        nets[0].rebuild([sp.seed for sp in specs])
        for i, net in enumerate(nets):
            got = net.to_host()
            for f in fields:
                np.testing.assert_array_equal(got[f], first[i][f], err_msg=f"replay {i} {f}")
    finally:
        for net in reversed(nets):
            net.close()


def test_graph_rebuild_of_seed_dependent_counts(snc, oracle_mod):
    """Every rule in a graph build: pairwise_bernoulli totals (capacity and
    padding) and fixed_total_number redraws (device-counted rounds) change
    with the seed at every replay."""
    specs = [
        W.two_population(333, "pairwise_bernoulli", p=0.05, autapses=False, seed=2),
        W.two_population(500, "fixed_total_number", k=40_000, autapses=False, multapses=False, seed=3),
        W.two_population(700, "fixed_indegree", k=31, autapses=False, seed=1),
        W.two_population(256, "pairwise_bernoulli", p=0.2, autapses=True, seed=4),  # 512 nodes: 2^9
        W.two_population(300, "fixed_total_number", k=20_000, autapses=False, multapses=True, seed=5),
        W.two_population(90, "all_to_all", autapses=False, seed=6),
    ] + W.batched_sweep(count=6, scale=0.05)
    _graph_trials(snc, oracle_mod, specs, (1000, 2000), oracle_members=(0, 1, 3))


@pytest.mark.parametrize("spec", [
    W.two_population(512, "pairwise_bernoulli", p=0.03, autapses=False, seed=41),
    W.two_population(400, "fixed_total_number", k=30_000, autapses=False, multapses=False, seed=42),
], ids=["bernoulli", "total_nomult"])
def test_graph_rebuild_single_network(snc, oracle_mod, spec):
    """A graph build of one network (digit counts fused in generation,
    padding counted by its own kernel)."""
    _graph_trials(snc, oracle_mod, [spec], (1000, 2000), oracle_members=(0,))


def test_graph_build_refuses_what_it_cannot_replay(snc):
    # A fixed_total_number without multapses taking almost every pair would
    # need more than 512 device-counted rounds.
    dense = W.two_population(40, "fixed_total_number", k=1500, autapses=False, multapses=False, seed=2)
    with pytest.raises(snc.SncError) as e:
        snc.Network.batch_graph([W.plain_indegree(n=50, k=5), dense])
    assert e.value.name == "UNSUPPORTED"
    net = snc.Network(W.plain_indegree(n=50, k=5)).finalize()
    with pytest.raises(snc.SncError) as e:
        net.rebuild([1])
    assert e.value.name == "STATE"
    net.close()


def test_batch_above_2_pow_30_positions_matches_single_builds(snc):
    """A batch whose arrays hold more than 2^30 connections (the per-segment
    sort must not fall back to a whole-array sort)."""
    specs = [W.two_population(100_000, "fixed_indegree", k=1400, seed=s) for s in (71, 72)]
    nets = snc.Network.batch(specs)
    assert sum(int(n.view().n_syn) for n in nets) > (1 << 30)
    for i, (spec, net) in enumerate(zip(specs, nets)):
        t = net.tensors()
        single = snc.Network(spec).finalize()
        r = single.tensors()
        for f in ("row_ptr", "group_ptr", "target", "delay", "weight", "group_first"):
            assert bool((t[f] == r[f]).all()), (i, f)
        single.close()
    for net in reversed(nets):
        net.close()


def test_graph_built_networks_free_call_buffers(snc):
    """A graph-built batch keeps its build buffers for the replays, but host
    copies and spike delivery on its members free their own temporaries:
    repeated calls leave the peak of live device memory where the first
    call put it."""
    import torch
    specs, _ = _fixed_count_specs()
    nets = snc.Network.batch_graph(specs)
    try:
        net = nets[0]
        t = net.tensors()
        gp = t["group_ptr"]
        src = torch.nonzero(gp[1:] > gp[:-1]).flatten().to(torch.int32)  # sources with a group
        grp = torch.zeros_like(src)
        mult = torch.ones(src.numel(), dtype=torch.float32, device=src.device)
        inp = torch.zeros(int(net.view().n_nodes), dtype=torch.float32, device=src.device)
        peaks = []
        for _ in range(3):
            torch.cuda.synchronize()
            net.to_host()
            net.deliver(src, grp, mult, inp)
            net.synchronize()
            peaks.append(int(net.stats().device_bytes_peak))
        assert peaks[0] == peaks[1] == peaks[2], peaks
        assert float(inp.abs().sum()) > 0
    finally:
        for net in reversed(nets):
            net.close()


def test_graph_replay_past_its_bounds_is_reported(snc, oracle_mod):
    """A replay that draws more Bernoulli connections than a projection's
    recorded capacity, or that still has redraws pending after the recorded
    rounds, is reported at the next synchronize (UNSUPPORTED, TIMEOUT) and
    writes nothing outside the build's arrays; the replays that stay inside
    their bounds give the single build's network.  The capacities are made
    small (mean + 1 sd) with the test hook, and the oracle's per-projection
    totals say in advance which seeds exceed them."""
    import math
    from dataclasses import replace
    n, p = 300, 0.05
    spec = W.two_population(n, "pairwise_bernoulli", p=p, autapses=False, seed=21)
    pairs = n * n
    cap = min(pairs, math.ceil(pairs * p + 1.0 * math.sqrt(pairs * p * (1.0 - p))))
    fields = ("src", "tgt", "delay", "weight", "row_ptr", "group_ptr", "group_first")

    def exceeds(seed):
        ref = oracle_mod.build(replace(spec, seed=seed))
        s, t = ref["src"].astype(np.int64), ref["tgt"].astype(np.int64)
        counts = [int(np.sum((s // n == a) & (t // n == b))) for a in (0, 1) for b in (0, 1)]
        return max(counts) > cap

    try:
        snc.snc_set_graph_test(1.0, 0.0, 0)
        nets = snc.Network.batch_graph([spec])
        outcomes = set()
        for seed in range(100, 112):
            nets[0].rebuild([seed])
            over = exceeds(seed)
            outcomes.add(over)
            if over:
                with pytest.raises(snc.SncError) as e:
                    nets[0].synchronize()
                assert e.value.name == "UNSUPPORTED", seed
            else:
                got = nets[0].to_host()
                single = snc.Network(replace(spec, seed=seed)).finalize()
                alone = single.to_host()
                single.close()
                for f in fields:
                    np.testing.assert_array_equal(got[f], alone[f], err_msg=f"seed {seed} {f}")
        assert outcomes == {True, False}  # both kinds of replay were exercised
        nets[0].close()
        # One redraw round for a total-number call that takes half of the pairs.
        snc.snc_set_graph_test(10.0, 32.0, 1)
        dense = W.two_population(100, "fixed_total_number", k=5_000, autapses=False, multapses=False, seed=23)
        nets = snc.Network.batch_graph([dense])
        with pytest.raises(snc.SncError) as e:
            nets[0].synchronize()
        assert e.value.name == "TIMEOUT"
        nets[0].close()
    finally:
        snc.snc_set_graph_test()
    # Back to the recorded defaults: the same networks build and replay correctly.
    nets = snc.Network.batch_graph([spec])
    nets[0].rebuild([101])
    got = nets[0].to_host()
    nets[0].close()
    assert_network_equal(got, oracle_mod.build(replace(spec, seed=101)), "defaults again")


def test_graph_rebuild_degenerate_members(snc, oracle_mod):
    """Graph builds with members that test the capacity and padding edges: a
    network with no projections, Bernoulli with p = 0 (a capacity of padding
    only) and p = 1 (the capacity is every pair), a power-of-two node count,
    one_to_one and a zero-count total-number call."""
    specs = [
        NetworkSpec(seed=51, dt=0.1, populations=[7], projections=[]),
        W.two_population(64, "pairwise_bernoulli", p=0.0, autapses=False, seed=52),
        W.two_population(32, "pairwise_bernoulli", p=1.0, autapses=False, seed=53),
        W.two_population(128, "pairwise_bernoulli", p=0.1, autapses=True, seed=54),
        W.two_population(40, "one_to_one", seed=55),
        W.two_population(30, "fixed_total_number", k=0, autapses=False, multapses=False, seed=56),
    ]
    _graph_trials(snc, oracle_mod, specs, (700,), oracle_members=(1, 2, 3))

"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Integer results (sources, targets, delay steps, CSR and group offsets) must be
bit-exact; weights within 4 fp32 ulp.  Sizes span several generation, sort
and index tiles and end in ragged tails.
"""
import numpy as np
import pytest

from gpu_helpers import assert_network_equal
from paper_2306_09855_gb300 import workloads as W
from paper_2306_09855_gb300.workloads import Dist, NetworkSpec, Projection

pytestmark = pytest.mark.gpu

WD = dict(weight=Dist("normal", 1.0, 0.1), delay=Dist("normal", 1.5, 0.75))


@pytest.fixture(scope="module")
def snc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09855_gb300 import snc as mod
    mod.load()
    return mod


def build_both(snc, oracle_mod, spec):
    net = snc.Network(spec).finalize()
    got = net.to_host()
    net.close()
    return got, oracle_mod.build(spec)


def test_plain_indegree_400k(snc, oracle_mod):
    spec = W.plain_indegree()
    got, ref = build_both(snc, oracle_mod, spec)
    assert ref["src"].size == 400_000
    assert_network_equal(got, ref, "plain")


RULES = [("fixed_indegree", dict(k=37)), ("fixed_outdegree", dict(k=41)),
         ("fixed_total_number", dict(k=250_003)), ("pairwise_bernoulli", dict(p=0.013)),
         ("all_to_all", {}), ("one_to_one", {})]


@pytest.mark.parametrize("rule,kw", RULES, ids=[r for r, _ in RULES])
@pytest.mark.parametrize("mult", [True, False], ids=["mult", "nomult"])
def test_rules_two_population(snc, oracle_mod, rule, kw, mult):
    n = 700 if rule == "all_to_all" else 3001
    spec = W.two_population(n, rule, autapses=mult, multapses=mult, seed=77, **kw)
    got, ref = build_both(snc, oracle_mod, spec)
    assert_network_equal(got, ref, f"{rule}/{mult}")


@pytest.mark.parametrize("aut,mult", [(True, False), (False, True)])
def test_mixed_flags(snc, oracle_mod, aut, mult):
    spec = NetworkSpec(seed=5, dt=0.1, populations=[900, 1100], projections=[
        Projection(src=(0, 900), tgt=(0, 2000), rule="fixed_indegree", k=60, autapses=aut, multapses=mult, **WD),
        Projection(src=(0, 2000), tgt=(450, 900), rule="fixed_outdegree", k=33, autapses=aut, multapses=mult, **WD),
        Projection(src=(100, 1500), tgt=(0, 2000), rule="fixed_total_number", k=123_457, autapses=aut,
                   multapses=mult, **WD),
        Projection(src=(0, 2000), tgt=(1000, 1000), rule="pairwise_bernoulli", p=0.02, autapses=aut, **WD),
        Projection(src=(10, 300), tgt=(200, 400), rule="all_to_all", autapses=aut, **WD),
    ])
    got, ref = build_both(snc, oracle_mod, spec)
    assert_network_equal(got, ref, "mixed")


def test_microcircuit_scaled(snc, oracle_mod):
    spec = W.microcircuit(scale=0.08)
    got, ref = build_both(snc, oracle_mod, spec)
    assert ref["src"].size > 1_000_000
    assert_network_equal(got, ref, "microcircuit")


def test_complement_and_dense_sampling(snc, oracle_mod):
    spec = NetworkSpec(seed=3, dt=0.1, populations=[64, 2000], projections=[
        Projection(src=(0, 64), tgt=(64, 2000), rule="fixed_indegree", k=50, multapses=False, **WD),
        Projection(src=(0, 64), tgt=(0, 64), rule="fixed_indegree", k=63, autapses=False, multapses=False, **WD),
        Projection(src=(0, 64), tgt=(64, 2000), rule="pairwise_bernoulli", p=0.9, **WD),
        Projection(src=(64, 2000), tgt=(0, 64), rule="fixed_outdegree", k=64, multapses=False, **WD),
    ])
    got, ref = build_both(snc, oracle_mod, spec)
    assert_network_equal(got, ref, "complement")


def test_edge_cases(snc, oracle_mod):
    cases = [
        NetworkSpec(seed=1, dt=0.1, populations=[10], projections=[]),
        NetworkSpec(seed=1, dt=0.1, populations=[10], projections=[
            Projection(src=(0, 10), tgt=(0, 10), rule="one_to_one", autapses=False, **WD)]),
        NetworkSpec(seed=1, dt=0.1, populations=[1, 1], projections=[
            Projection(src=(0, 1), tgt=(1, 1), rule="one_to_one", **WD)]),
        NetworkSpec(seed=1, dt=0.1, populations=[5, 7], projections=[
            Projection(src=(0, 5), tgt=(5, 7), rule="pairwise_bernoulli", p=0.0, **WD),
            Projection(src=(0, 5), tgt=(5, 7), rule="pairwise_bernoulli", p=1.0, **WD),
            Projection(src=(0, 5), tgt=(5, 7), rule="fixed_indegree", k=0, **WD)]),
        # sources with no outgoing connections, constant delays, big delays
        NetworkSpec(seed=2, dt=0.25, populations=[5000, 3], projections=[
            Projection(src=(4990, 10), tgt=(5000, 3), rule="fixed_indegree", k=9000,
                       weight=Dist("const", -2.5), delay=Dist("const", 1000.0)),
            Projection(src=(0, 3), tgt=(5000, 3), rule="all_to_all", weight=Dist("const", 1.0),
                       delay=Dist("normal", 40.0, 10.0))]),
        # delay below one step everywhere
        NetworkSpec(seed=9, dt=1.0, populations=[50], projections=[
            Projection(src=(0, 50), tgt=(0, 50), rule="fixed_total_number", k=999,
                       weight=Dist("normal", 0.0, 1.0), delay=Dist("normal", 0.01, 0.001))]),
    ]
    for i, spec in enumerate(cases):
        got, ref = build_both(snc, oracle_mod, spec)
        assert_network_equal(got, ref, f"edge{i}")


BAD = [
    Projection(src=(0, 3), tgt=(3, 4), rule="one_to_one", **WD),
    Projection(src=(0, 3), tgt=(3, 4), rule="fixed_indegree", k=4, multapses=False, **WD),
    Projection(src=(0, 3), tgt=(0, 3), rule="fixed_indegree", k=3, autapses=False, multapses=False, **WD),
    Projection(src=(0, 1), tgt=(0, 1), rule="fixed_total_number", k=1, autapses=False, **WD),
    Projection(src=(0, 2), tgt=(2, 2), rule="fixed_total_number", k=5, multapses=False, **WD),
    Projection(src=(0, 3), tgt=(5, 4), rule="all_to_all", **WD),
    Projection(src=(0, 3), tgt=(3, 4), rule="pairwise_bernoulli", p=1.5, **WD),
]


@pytest.mark.parametrize("proj", BAD)
def test_connect_errors_match_oracle(snc, oracle_mod, proj):
    spec = NetworkSpec(seed=1, dt=0.1, populations=[3, 4], projections=[proj])
    expect = oracle_mod.STATUS[oracle_mod.check_projection(spec, 0)]
    with pytest.raises(snc.SncError) as e:
        snc.Network(spec)
    assert e.value.name == expect


def test_connect_after_finalize_is_state_error(snc):
    spec = W.plain_indegree(n=50, k=5)
    net = snc.Network(spec).finalize()
    pj = spec.projections[0]
    with pytest.raises(snc.SncError) as e:
        snc.snc_connect(net.ctx, snc.snc_range(*pj.src), snc.snc_range(*pj.tgt),
                        snc._rule_struct(pj), snc._syn_struct(pj))
    assert e.value.name == "STATE"
    net.close()


def test_launch_shape_independence(snc):
    """Two builds of one spec are identical (grid / block shapes do not
    enter the draws); a different seed changes the network."""
    spec = W.two_population(2000, "fixed_total_number", k=300_000, seed=11)
    a = snc.Network(spec).finalize().to_host()
    b = snc.Network(spec).finalize().to_host()
    for f in ("src", "tgt", "delay", "weight"):
        np.testing.assert_array_equal(a[f], b[f])


@pytest.mark.parametrize("digit_bits,group,items", [(11, 8, 16), (8, 0, 16), (9, 4, 16), (8, 0, 12), (9, 0, 8),
                                                   (9, 0, 32), (8, 0, 24)],
                         ids=["d11g8", "d8tma", "d9g4", "d8tma_i12", "d9tma_i8", "d9tma_i32", "d8tma_i24"])
@pytest.mark.parametrize("n_nodes,delay", [(4, Dist("const", 0.1)), (60, Dist("normal", 1.5, 0.75)),
                                           (3000, Dist("normal", 1.5, 0.75)),
                                           (600_000, Dist("normal", 1.5, 0.75)),
                                           (140_000, Dist("const", 6000.0))],
                         ids=["3bit", "12bit", "18bit", "26bit", "34bit_wide"])
def test_every_pass_parity(snc, oracle_mod, n_nodes, delay, digit_bits, group, items):
    """The sort's buffers alternate per pass, so the result buffer depends on
    the parity of the pass count: cover odd and even counts for every kernel
    variant (1-4 passes of 8 bits on 32-bit keys, and a 34-bit key that
    takes the 64-bit key path: 60,000 delay steps need 16 bits)."""
    half = n_nodes // 2
    spec = NetworkSpec(seed=21, dt=0.1, populations=[half, n_nodes - half], projections=[
        Projection(src=(0, n_nodes), tgt=(0, n_nodes), rule="fixed_total_number", k=150_001,
                   weight=Dist("normal", 5.0, 1.0), delay=delay)])
    old = snc.snc_get_tuning()
    try:
        snc.snc_set_tuning(sort_digit_bits=digit_bits, sort_group_tiles=group, sort_items=items)
        net = snc.Network(spec).finalize()
        got = net.to_host()
        st = net.stats()
        net.close()
    finally:
        snc.snc_set_tuning(sort_digit_bits=old.sort_digit_bits, sort_group_tiles=old.sort_group_tiles,
                           sort_items=old.sort_items)
    assert st.n_passes == -(-st.key_bits // digit_bits)
    assert_network_equal(got, oracle_mod.build(spec), f"passes={st.n_passes}")


def test_copy_index_and_network_copy_match_views(snc):
    spec = W.two_population(3000, "fixed_indegree", k=50, autapses=False, seed=41)
    net = snc.Network(spec).finalize()
    full = net.to_host()
    v = net.view()
    n, nn, ng = int(v.n_syn), int(v.n_nodes), int(v.n_groups)
    out = {"tgt": np.empty(n, np.uint32), "delay": np.empty(n, np.uint16), "weight": np.empty(n, np.float32),
           "row_ptr": np.empty(nn + 1, np.uint64), "group_ptr": np.empty(nn + 1, np.uint64),
           "group_first": np.empty(ng + 5, np.uint64)}
    assert net.to_host_network(out) == n
    for f in ("tgt", "delay", "weight", "row_ptr", "group_ptr"):
        np.testing.assert_array_equal(out[f].astype(full[f].dtype), full[f], err_msg=f)
    np.testing.assert_array_equal(out["group_first"][:ng], full["group_first"][:ng])
    src = np.repeat(np.arange(nn, dtype=np.uint32), np.diff(out["row_ptr"].astype(np.int64)))
    np.testing.assert_array_equal(src, full["src"])
    small = np.empty(max(1, ng - 1), np.uint64)
    status = snc.load().snc_copy_index(net.ctx, out["row_ptr"].ctypes.data, out["group_ptr"].ctypes.data,
                                       small.ctypes.data, small.size)
    assert status == snc.SNC_ERR_INVALID_ARG
    net.close()


def test_async_network_copy_while_another_builds(snc):
    """snc_copy_network_async: network A's copies are queued into page-locked
    arrays while network B is finalized on another stream; after A's
    synchronize the arrays equal the synchronous copies, and a refused
    capacity queues nothing."""
    torch = pytest.importorskip("torch")
    spec_a = W.two_population(3000, "fixed_indegree", k=50, autapses=False, seed=42)
    spec_b = W.two_population(4000, "pairwise_bernoulli", p=0.02, seed=43)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    a = snc.Network(spec_a, stream=sa).finalize()
    ref = a.to_host()
    v = a.view()
    n, nn, ng = int(v.n_syn), int(v.n_nodes), int(v.n_groups)

    def pinned(count, dt):
        return torch.empty(max(1, count), dtype=dt, pin_memory=True).numpy()

    out = {"tgt": pinned(n, torch.int32).view(np.uint32), "delay": pinned(n, torch.int16).view(np.uint16),
           "weight": pinned(n, torch.float32), "row_ptr": pinned(nn + 1, torch.int64).view(np.uint64),
           "group_ptr": pinned(nn + 1, torch.int64).view(np.uint64),
           "group_first": pinned(ng, torch.int64).view(np.uint64)}
    for arr in out.values():
        arr.fill(0xFF if arr.dtype != np.float32 else 0)
    small = dict(out, group_first=out["group_first"][:max(0, ng - 1)])
    with pytest.raises(Exception):
        a.to_host_network(small, wait=False)
    status = snc.load().snc_copy_network_async(a.ctx, out["tgt"].ctypes.data, out["delay"].ctypes.data,
                                              out["weight"].ctypes.data, n - 1, 0, 0, 0, 0)
    assert status == snc.SNC_ERR_INVALID_ARG
    assert a.to_host_network(out, wait=False) == n
    b = snc.Network(spec_b, stream=sb).finalize()
    a.synchronize()
    for f in ("tgt", "delay", "weight", "row_ptr", "group_ptr"):
        np.testing.assert_array_equal(out[f].astype(ref[f].dtype), ref[f], err_msg=f)
    np.testing.assert_array_equal(out["group_first"][:ng], ref["group_first"][:ng])
    b.synchronize()
    assert int(b.view().n_syn) > 0
    b.close()
    a.close()


def test_redraw_super_buckets(snc, oracle_mod):
    """fixed_total_number without multapses above 2^19 slots: round-0 pairs
    pass through several super-buckets before their buckets (1.5e6 slots on
    1e7 pairs, so that many slots redraw over several rounds), next to a
    projection that redraws autapses only."""
    spec = NetworkSpec(seed=29, dt=0.1, populations=[2500, 1500], projections=[
        Projection(src=(0, 2500), tgt=(0, 4000), rule="fixed_total_number", k=1_500_000, autapses=False,
                   multapses=False, weight=Dist("normal", 8.0, 1.0), delay=Dist("normal", 1.5, 0.75)),
        Projection(src=(2500, 1500), tgt=(0, 2500), rule="fixed_total_number", k=700_001, multapses=False,
                   weight=Dist("normal", -3.0, 0.4), delay=Dist("normal", 1.5, 0.75)),
        Projection(src=(0, 4000), tgt=(0, 4000), rule="fixed_total_number", k=600_000, autapses=False,
                   weight=Dist("normal", 2.0, 0.25), delay=Dist("normal", 1.5, 0.75))])
    net = snc.Network(spec).finalize()
    got = net.to_host()
    net.close()
    assert_network_equal(got, oracle_mod.build(spec), "super-buckets")


def _build_with_stats(snc, spec):
    net = snc.Network(spec).finalize()
    got = net.to_host()
    st = net.stats()
    net.close()
    return got, st


@pytest.mark.parametrize("aut,mult", [(True, True), (False, False), (False, True)], ids=["both", "neither", "mult"])
def test_source_major_sort(snc, oracle_mod, aut, mult):
    """Builds made only of rules that generate source by source (one_to_one,
    all_to_all, fixed_outdegree) take the per-source counting sort by delay
    step: sources shared by several projections, rows longer than one chunk
    (all_to_all on 3,000 targets), the one_to_one projection that drops all
    its pairs, and the same result as the oracle's stable sort."""
    WD = dict(weight=Dist("normal", 20.0, 1.0), delay=Dist("normal", 1.5, 0.75))
    spec = NetworkSpec(seed=33, dt=0.1, populations=[1000, 3000, 500], projections=[
        Projection(src=(0, 1000), tgt=(1000, 3000), rule="all_to_all", autapses=aut, multapses=mult, **WD),
        Projection(src=(0, 4500), tgt=(0, 4500), rule="fixed_outdegree", k=37, autapses=aut, multapses=mult, **WD),
        Projection(src=(1000, 500), tgt=(4000, 500), rule="one_to_one", autapses=aut, multapses=mult, **WD),
        Projection(src=(4000, 500), tgt=(4000, 500), rule="one_to_one", autapses=aut, multapses=mult, **WD),
        Projection(src=(500, 1000), tgt=(0, 1500), rule="all_to_all", autapses=aut, multapses=mult, **WD),
        Projection(src=(4000, 500), tgt=(3000, 1500), rule="fixed_outdegree", k=1200, autapses=aut,
                   multapses=mult, **WD)])
    got, st = _build_with_stats(snc, spec)
    assert st.source_major == 1 and st.n_passes == 0
    assert_network_equal(got, oracle_mod.build(spec), "source-major")


@pytest.mark.parametrize("delay", [Dist("const", 0.1), Dist("normal", 25.0, 3.0)], ids=["one_step", "nine_bits"])
def test_source_major_delay_widths(snc, oracle_mod, delay):
    """The per-source sort at the narrowest delay field (a single delay step:
    one bit) and at the widest it takes (nine bits), with sources of one chunk
    and of several."""
    WD = dict(weight=Dist("normal", 20.0, 1.0), delay=delay)
    spec = NetworkSpec(seed=36, dt=0.1, populations=[700, 2600], projections=[
        Projection(src=(0, 700), tgt=(700, 2600), rule="fixed_outdegree", k=300, **WD),
        Projection(src=(0, 300), tgt=(700, 2600), rule="all_to_all", **WD)])
    got, st = _build_with_stats(snc, spec)
    assert st.source_major == 1 and st.n_passes == 0
    if delay.kind == "normal":
        assert int(got["delay"].max()) >= 256
    assert_network_equal(got, oracle_mod.build(spec), "source-major delay width")


def test_source_major_falls_back(snc, oracle_mod):
    """A fixed_indegree projection in the build, or delays beyond 9 bits, keep
    the radix sort."""
    WD = dict(weight=Dist("normal", 20.0, 1.0), delay=Dist("normal", 1.5, 0.75))
    mixed = NetworkSpec(seed=34, dt=0.1, populations=[800, 800], projections=[
        Projection(src=(0, 800), tgt=(800, 800), rule="all_to_all", **WD),
        Projection(src=(800, 800), tgt=(0, 800), rule="fixed_indegree", k=40, **WD)])
    got, st = _build_with_stats(snc, mixed)
    assert st.source_major == 0 and st.n_passes >= 1
    assert_network_equal(got, oracle_mod.build(mixed), "mixed rules")
    wide = NetworkSpec(seed=35, dt=0.1, populations=[600, 600], projections=[
        Projection(src=(0, 600), tgt=(600, 600), rule="fixed_outdegree", k=50, weight=Dist("normal", 6.0, 1.0),
                   delay=Dist("const", 100.0))])
    got, st = _build_with_stats(snc, wide)
    assert st.source_major == 0
    assert_network_equal(got, oracle_mod.build(wide), "wide delays")


def test_sparse_samplers_wide_ranges(snc, oracle_mod):
    """Selections without replacement of at most 100 of 20,000-60,000
    candidates (in-degree, out-degree with the autapse skip, Bernoulli
    subsets) in one build: the oracle's sequential rule exactly."""
    WD = dict(weight=Dist("normal", 20.0, 1.0), delay=Dist("normal", 1.5, 0.75))
    spec = NetworkSpec(seed=44, dt=0.1, populations=[60_000, 20_000], projections=[
        Projection(src=(0, 60_000), tgt=(60_000, 20_000), rule="fixed_indegree", k=90, multapses=False, **WD),
        Projection(src=(0, 60_000), tgt=(0, 60_000), rule="fixed_outdegree", k=25, autapses=False,
                   multapses=False, **WD),
        Projection(src=(60_000, 20_000), tgt=(0, 30_000), rule="pairwise_bernoulli", p=0.002, **WD)])
    got, _ = _build_with_stats(snc, spec)
    assert_network_equal(got, oracle_mod.build(spec), "sparse samplers")


def test_device_counted_redraw_rounds(snc, oracle_mod):
    """A plain fixed_total_number build without multapses that needs few
    rounds counts them on the device: with the default number it equals the
    oracle; held to one round by the test hook (about a fifth of the pairs
    taken, so hundreds of slots still pending) it reports TIMEOUT at the next
    synchronize instead of returning a wrong network; the build after the
    reset is the oracle's again."""
    spec = W.two_population(300, "fixed_total_number", k=20_000, autapses=False, multapses=False, seed=24)
    got = snc.Network(spec).finalize()
    assert_network_equal(got.to_host(), oracle_mod.build(spec), "device-counted rounds")
    got.close()
    try:
        snc.snc_set_graph_test(10.0, 32.0, 1)
        net = snc.Network(spec)
        with pytest.raises(snc.SncError) as e:
            net.finalize()
            net.synchronize()
        assert e.value.name == "TIMEOUT"
        net.close()
    finally:
        snc.snc_set_graph_test(10.0, 32.0, 0)
    again = snc.Network(spec).finalize()
    assert_network_equal(again.to_host(), oracle_mod.build(spec), "after the reset")
    again.close()


def test_redraw_global_tables(snc, oracle_mod):
    """fixed_total_number without multapses on node ranges too wide for a
    packed (pair, slot) word (2 x 2.1e6 nodes, 1.1e6 slots: 68 bits) takes the
    global pair tables instead of buckets; same network as the oracle."""
    WD = dict(weight=Dist("normal", 20.0, 1.0), delay=Dist("normal", 1.5, 0.75))
    spec = NetworkSpec(seed=45, dt=0.1, populations=[2_100_000, 2_100_000], projections=[
        Projection(src=(0, 4_200_000), tgt=(0, 4_200_000), rule="fixed_total_number", k=1_100_000,
                   autapses=False, multapses=False, **WD),
        Projection(src=(0, 1000), tgt=(0, 1000), rule="fixed_total_number", k=200_000, autapses=False, **WD)])
    got, _ = _build_with_stats(snc, spec)
    assert_network_equal(got, oracle_mod.build(spec), "global tables")

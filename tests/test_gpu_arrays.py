"""Explicit node-id arrays and per-connection weight/delay arrays in Connect
(Sec. 2.1) on the GPU (snc_connect_arrays) against the oracle's array
networks, element by element: every rule and autapse/multapse pair, ids on
one side or both, repeated ids where the rule allows them, the weight
array 0, 1, 2, ... that exposes the Sec. 2.1 connection numbering, delays
given in ms, a batch and a network spanning many tiles."""
import numpy as np
import pytest

from gpu_helpers import assert_network_equal
from paper_2306_09855_gb300.workloads import Dist, NetworkSpec, Projection

pytestmark = pytest.mark.gpu

WD = dict(weight=Dist("normal", 1.0, 0.1), delay=Dist("normal", 1.5, 0.75))
FLAGS = [(True, True), (False, True), (True, False), (False, False)]  # (autapses, multapses)
RULES = ["one_to_one", "all_to_all", "fixed_indegree", "fixed_outdegree", "fixed_total_number",
         "pairwise_bernoulli"]


@pytest.fixture(scope="module")
def snc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09855_gb300 import snc as mod
    mod.load()
    return mod


def _build(snc, spec):
    net = snc.Network(spec).finalize()
    got = net.to_host()
    net.close()
    return got


def _numbered(rule, ns, nt, k):
    return {"one_to_one": ns, "all_to_all": ns * nt, "fixed_indegree": nt * k, "fixed_outdegree": ns * k,
            "fixed_total_number": k}.get(rule, 0)


def _proj(rule, aut, mult, src_ids, tgt_ids, rng, weights="draw", delays="draw", k=None):
    ns = len(src_ids) if src_ids is not None else 300
    nt = len(tgt_ids) if tgt_ids is not None else (ns if rule == "one_to_one" else 250)
    kw = {"fixed_indegree": dict(k=k or 29), "fixed_outdegree": dict(k=k or 31),
          "fixed_total_number": dict(k=k or 20_011), "pairwise_bernoulli": dict(p=0.05)}.get(rule, {})
    n = _numbered(rule, ns, nt, kw.get("k", 0))
    extra = {}
    if weights == "numbers" and n:
        extra["weights"] = np.arange(n, dtype=np.float32)
    elif weights == "random" and n:
        extra["weights"] = rng.normal(3.0, 0.5, n).astype(np.float32)
    if delays == "random" and n:
        extra["delays"] = rng.uniform(0.05, 4.0, n).astype(np.float32)
    return Projection(src=(0 if src_ids is not None else 40, ns), tgt=(0 if tgt_ids is not None else 100, nt),
                      rule=rule, autapses=aut, multapses=mult, src_ids=src_ids, tgt_ids=tgt_ids, **kw, **WD,
                      **extra)


@pytest.mark.parametrize("aut,mult", FLAGS)
@pytest.mark.parametrize("rule", RULES)
def test_lists_on_both_sides(snc, oracle_mod, rule, aut, mult):
    rng = np.random.default_rng(hash((rule, aut, mult)) % 2**32)
    perm = rng.permutation(700).astype(np.uint32)
    src_ids = perm[:300]
    tgt_ids = perm[150:150 + (300 if rule == "one_to_one" else 250)]  # overlap: autapse pairs exist
    arrays = rule != "pairwise_bernoulli"
    pj = _proj(rule, aut, mult, src_ids, tgt_ids, rng, weights="random" if arrays else "draw",
               delays="random" if arrays else "draw")
    spec = NetworkSpec(seed=7, dt=0.1, populations=[400, 300], projections=[pj])
    ref = oracle_mod.build(spec)
    assert ref["src"].size > 0
    assert_network_equal(_build(snc, spec), ref, f"{rule}/{aut}/{mult}")


@pytest.mark.parametrize("aut,mult", FLAGS)
@pytest.mark.parametrize("rule", RULES)
def test_list_on_one_side_and_numbered_weights(snc, oracle_mod, rule, aut, mult):
    """Sources as a list, targets as a range (and the reverse for half the
    rules); weights 0, 1, 2, ... give each connection its number."""
    rng = np.random.default_rng(11)
    ids = rng.permutation(600).astype(np.uint32)[:300]
    if rule in ("fixed_outdegree", "all_to_all", "fixed_total_number"):
        pj = _proj(rule, aut, mult, None, ids[:250], rng, weights="numbers")
    else:
        pj = _proj(rule, aut, mult, ids, None, rng, weights="numbers" if rule != "pairwise_bernoulli" else "draw")
    spec = NetworkSpec(seed=12, dt=0.1, populations=[600], projections=[pj])
    assert_network_equal(_build(snc, spec), oracle_mod.build(spec), f"{rule}/{aut}/{mult}")


@pytest.mark.parametrize("rule", ["one_to_one", "all_to_all", "fixed_indegree", "fixed_total_number"])
def test_repeated_ids_where_allowed(snc, oracle_mod, rule):
    """Multapses allowed and autapses off: lists may repeat ids (one_to_one
    and all_to_all then drop every equal pair; the in-degree rule's source
    list must stay distinct, so only its targets repeat)."""
    rng = np.random.default_rng(5)
    src_ids = rng.integers(0, 120, 300).astype(np.uint32)
    tgt_ids = rng.integers(0, 120, 300 if rule == "one_to_one" else 260).astype(np.uint32)
    if rule == "fixed_indegree":
        src_ids = rng.permutation(120).astype(np.uint32)
    pj = _proj(rule, False, True, src_ids, tgt_ids, rng, weights="numbers", delays="random")
    spec = NetworkSpec(seed=3, dt=0.1, populations=[120], projections=[pj])
    assert_network_equal(_build(snc, spec), oracle_mod.build(spec), rule)


def test_many_tiles_and_mixed_calls(snc, oracle_mod):
    """Array calls beside range calls in one network large enough for
    several generation chunks and sort tiles (ragged tails)."""
    rng = np.random.default_rng(8)
    perm = rng.permutation(20_000).astype(np.uint32)
    projs = [
        _proj("fixed_indegree", False, False, perm[:9000], perm[5000:17000], rng, weights="random", k=40),
        Projection(src=(0, 20_000), tgt=(0, 20_000), rule="fixed_outdegree", k=17, autapses=False, **WD),
        _proj("fixed_total_number", False, False, perm[3000:15000], perm[:11000], rng, delays="random",
              k=300_001),
        _proj("all_to_all", False, True, perm[100:700], perm[300:1100], rng, weights="numbers"),
        _proj("pairwise_bernoulli", False, True, perm[:5000], perm[2000:4000], rng),
    ]
    spec = NetworkSpec(seed=99, dt=0.1, populations=[12_000, 8_000], projections=projs)
    ref = oracle_mod.build(spec)
    assert ref["src"].size > 1_000_000
    assert_network_equal(_build(snc, spec), ref, "mixed")


def test_batch_members_with_arrays(snc, oracle_mod):
    rng = np.random.default_rng(2)
    specs = []
    for m in range(3):
        perm = rng.permutation(900).astype(np.uint32)
        specs.append(NetworkSpec(seed=40 + m, dt=0.1, populations=[900], projections=[
            _proj("fixed_indegree", False, False, perm[:400], perm[200:700], rng, weights="numbers", k=25),
            _proj("one_to_one", False, True, perm[:300], rng.permutation(900)[:300].astype(np.uint32), rng,
                  delays="random")]))
    nets = snc.Network.batch(specs)
    got = [n.to_host() for n in nets]
    for n in reversed(nets):
        n.close()
    for m, spec in enumerate(specs):
        assert_network_equal(got[m], oracle_mod.build(spec), f"member {m}")


def test_graph_rebuild_with_arrays(snc, oracle_mod):
    """A graph-recorded batch whose members connect through id lists and
    per-connection weight/delay arrays (with a Bernoulli and a no-multapse
    total-number call): each rebuild with new seeds equals the oracle's
    network for those seeds (the arrays are replayed from the recorded
    copies)."""
    from dataclasses import replace
    rng = np.random.default_rng(12)
    specs = []
    for m in range(3):
        perm = rng.permutation(900).astype(np.uint32)
        specs.append(NetworkSpec(seed=70 + m, dt=0.1, populations=[900], projections=[
            _proj("fixed_indegree", False, False, perm[:400], perm[200:700], rng, weights="numbers", k=25),
            _proj("pairwise_bernoulli", False, True, perm[:300], perm[100:400], rng),
            _proj("fixed_total_number", False, False, perm[:300], perm[300:600], rng, weights="random",
                  delays="random", k=9_000)]))
    nets = snc.Network.batch_graph(specs)
    try:
        for offset in (0, 500):
            seeds = [sp.seed + offset for sp in specs]
            if offset:
                nets[0].rebuild(seeds)
            for m, spec in enumerate(specs):
                assert_network_equal(nets[m].to_host(), oracle_mod.build(replace(spec, seed=seeds[m])),
                                     f"offset {offset} member {m}")
    finally:
        for n in reversed(nets):
            n.close()


def test_array_errors_match_the_oracle(snc, oracle_mod):
    """Connect refuses what the oracle's checks refuse, with the same status."""
    cases = [
        dict(src_ids=np.array([1, 2, 99], np.uint32)),                     # id above the nodes
        dict(src_ids=np.array([1, 2, 2], np.uint32), multapses=False),     # repeated id, multapses off
        dict(weights=np.ones(5, np.float32)),                              # wrong length
        dict(delays=np.array([1, 1, np.nan, 1, 1, 1, 1, 1, 1], np.float32)),
        dict(delays=np.full(9, 7000.0, np.float32)),                       # above 65535 steps
    ]
    for kw in cases:
        base = dict(src=(0, 3), tgt=(0, 3), rule="all_to_all", autapses=True, multapses=True, **WD)
        if "src_ids" in kw:
            base["src"] = (0, len(kw["src_ids"]))
        base.update(kw)
        spec = NetworkSpec(seed=1, dt=0.1, populations=[10], projections=[Projection(**base)])
        want = oracle_mod.STATUS[oracle_mod.check_projection(spec, 0)]
        assert want != "OK"
        with pytest.raises(snc.SncError) as e:
            snc.Network(spec)
        assert e.value.name == want, (kw, e.value.name, want)

"""Pin of the oracle's host-thread build (snc_oracle_par.c): it must give
the single-thread oracle's network bit for bit, so that full-size checks and
the multi-core CPU baseline use the pinned arithmetic.  Every rule and flag
pair, explicit arrays, several projections per network, empty and degenerate
projections, and thread counts from 1 up."""
import numpy as np
import pytest

from paper_2306_09855_gb300 import workloads as W
from paper_2306_09855_gb300.workloads import Dist, NetworkSpec, Projection

WD = dict(weight=Dist("normal", 1.0, 0.1), delay=Dist("normal", 1.5, 0.75))
FIELDS = ("src", "tgt", "delay", "weight", "row_ptr", "group_ptr", "group_first", "per_proj")
RULES = [("fixed_indegree", dict(k=23)), ("fixed_outdegree", dict(k=19)),
         ("fixed_total_number", dict(k=30_011)), ("pairwise_bernoulli", dict(p=0.03)),
         ("all_to_all", {}), ("one_to_one", {})]


def _same(oracle_mod, spec, threads=0):
    ref = oracle_mod.build(spec)
    got = oracle_mod.build_parallel(spec, threads)
    for f in FIELDS:
        np.testing.assert_array_equal(got[f], ref[f], err_msg=f)
    assert got["n_groups"] == ref["n_groups"]
    return ref


@pytest.mark.parametrize("aut,mult", [(True, True), (False, False), (True, False), (False, True)])
@pytest.mark.parametrize("rule,kw", RULES, ids=[r for r, _ in RULES])
def test_parallel_build_equals_single_thread(oracle_mod, rule, kw, aut, mult):
    n = 300 if rule == "all_to_all" else 1201
    spec = W.two_population(n, rule, autapses=aut, multapses=mult, seed=41, **kw)
    ref = _same(oracle_mod, spec)
    assert ref["src"].size > 0


@pytest.mark.parametrize("threads", [1, 2, 3, 7])
def test_thread_count_does_not_change_the_network(oracle_mod, threads):
    spec = NetworkSpec(seed=12, dt=0.1, populations=[700, 900], projections=[
        Projection(src=(0, 700), tgt=(0, 1600), rule="fixed_indegree", k=40, autapses=False, **WD),
        Projection(src=(0, 1600), tgt=(300, 600), rule="pairwise_bernoulli", p=0.05, autapses=False,
                   multapses=False, **WD),
        Projection(src=(100, 1200), tgt=(0, 1600), rule="fixed_total_number", k=50_000, autapses=False, **WD),
        Projection(src=(0, 1600), tgt=(0, 800), rule="fixed_outdegree", k=30, multapses=False, **WD),
        Projection(src=(10, 200), tgt=(100, 300), rule="all_to_all", autapses=False, **WD),
        Projection(src=(0, 500), tgt=(200, 500), rule="one_to_one", autapses=False, **WD),
    ])
    _same(oracle_mod, spec, threads)


def test_microcircuit_shape(oracle_mod):
    _same(oracle_mod, W.microcircuit(scale=0.02))


def test_explicit_arrays(oracle_mod):
    rng = np.random.default_rng(3)
    ids = rng.permutation(500).astype(np.uint32)
    projs = []
    for rule, kw in RULES:
        ns, nt = (60, 60) if rule == "one_to_one" else (60, 45)
        base = dict(src=(0, ns), tgt=(0, nt), rule=rule, autapses=False, multapses=False,
                    src_ids=ids[:ns], tgt_ids=ids[40:40 + nt], **WD)
        kw = dict(kw)
        if rule == "fixed_total_number":
            kw["k"] = 900
        count = {"one_to_one": ns, "all_to_all": ns * nt, "fixed_indegree": nt * kw.get("k", 0),
                 "fixed_outdegree": ns * kw.get("k", 0), "fixed_total_number": kw.get("k", 0)}.get(rule)
        if count:
            base["weights"] = rng.normal(2.0, 0.3, count).astype(np.float32)
            base["delays"] = rng.uniform(0.1, 3.0, count).astype(np.float32)
        projs.append(Projection(**base, **kw))
    _same(oracle_mod, NetworkSpec(seed=8, dt=0.1, populations=[500], projections=projs))


def test_empty_and_degenerate(oracle_mod):
    spec = NetworkSpec(seed=1, dt=0.1, populations=[50, 1], projections=[
        Projection(src=(0, 50), tgt=(0, 50), rule="fixed_indegree", k=0, **WD),
        Projection(src=(0, 50), tgt=(0, 50), rule="pairwise_bernoulli", p=0.0, **WD),
        Projection(src=(0, 50), tgt=(0, 50), rule="pairwise_bernoulli", p=1.0, autapses=False, **WD),
        Projection(src=(50, 1), tgt=(0, 51), rule="fixed_outdegree", k=51, multapses=False, **WD),
        Projection(src=(0, 0), tgt=(0, 50), rule="all_to_all", **WD),
        Projection(src=(0, 51), tgt=(0, 51), rule="fixed_total_number", k=0, **WD),
    ])
    _same(oracle_mod, spec)
    _same(oracle_mod, NetworkSpec(seed=1, dt=0.1, populations=[10], projections=[]))


@pytest.mark.parametrize("aut,mult,n", [(False, False, 1500), (True, False, 1599), (False, True, 20_000),
                                        (False, False, 1)])
def test_total_number_redraw_rounds(oracle_mod, aut, mult, n):
    """Dense fixed_total_number (almost every allowed pair taken): many
    redraw rounds, claims on the same pair within a round and across rounds;
    the threaded rounds pick the single-thread oracle's winners."""
    spec = NetworkSpec(seed=17, dt=0.1, populations=[40], projections=[
        Projection(src=(0, 40), tgt=(0, 40), rule="fixed_total_number", k=n, autapses=aut, multapses=mult, **WD)])
    _same(oracle_mod, spec, 3)

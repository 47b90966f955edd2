"""Pins of the oracle's explicit arrays in Connect (Sec. 2.1): node ids given
by arrays, the rule's index formulas then giving positions in the arrays,
and weights and delays given per connection by arrays as long as the number
of connections the rule numbers.

The pins tie the array forms to the range forms (pinned in
test_oracle_rules.py) through exact invariances, and to the paper's index
formulas through closed forms:
  * renaming every node by a bijection f commutes with the build, so
    arrays f[range] give f of the range build (autapse handling included);
  * with autapses and multapses allowed, any map g (repeats too) commutes;
  * a weight array holding 0, 1, 2, ... exposes each connection's number
    i_newconns, which the Sec. 2.1 formulas tie to its endpoints;
  * delays in ms become round(d / dt) steps, at least one (hand-computed
    values on a binary dt);
  * the complete cases (K = every candidate, N = every allowed pair) have
    one possible result.
"""
import itertools

import numpy as np
import pytest
from scipy import stats

from paper_2306_09855_gb300.workloads import Dist, NetworkSpec, Projection

WD = dict(weight=Dist("normal", 1.0, 0.1), delay=Dist("normal", 1.5, 0.75))
FLAGS = [(True, True), (False, True), (True, False), (False, False)]  # (autapses, multapses)


def net(n_nodes, projs, seed=99, dt=0.1):
    return NetworkSpec(seed=seed, dt=dt, populations=[n_nodes], projections=list(projs))


def rule_kw(rule):
    return {"fixed_indegree": dict(k=7), "fixed_outdegree": dict(k=7), "fixed_total_number": dict(k=900),
            "pairwise_bernoulli": dict(p=0.2)}.get(rule, {})


def range_proj(rule, aut, mult, src=(0, 40), tgt=(25, 40), **kw):
    if rule == "one_to_one":
        tgt = (tgt[0], src[1])
    return Projection(src=src, tgt=tgt, rule=rule, autapses=aut, multapses=mult, **rule_kw(rule), **WD, **kw)


def with_ids(pj, src_ids, tgt_ids):
    return Projection(src=(0, len(src_ids)), tgt=(0, len(tgt_ids)), rule=pj.rule, k=pj.k, p=pj.p,
                      autapses=pj.autapses, multapses=pj.multapses, weight=pj.weight, delay=pj.delay,
                      src_ids=np.asarray(src_ids, np.uint32), tgt_ids=np.asarray(tgt_ids, np.uint32),
                      weights=pj.weights, delays=pj.delays)


@pytest.mark.parametrize("aut,mult", FLAGS)
@pytest.mark.parametrize("rule", ["one_to_one", "all_to_all", "fixed_indegree", "fixed_outdegree",
                                  "fixed_total_number", "pairwise_bernoulli"])
def test_renaming_nodes_commutes_with_the_build(oracle_mod, rule, aut, mult):
    """Arrays f[range] for a bijection f of the node ids give f of the range
    build: positions, draws, autapse skips and redraws are unchanged."""
    n_nodes = 80
    base = range_proj(rule, aut, mult)
    f = np.random.default_rng(5).permutation(n_nodes).astype(np.uint32)
    s0, ns = base.src
    t0, nt = base.tgt
    ref = oracle_mod.generate(net(n_nodes, [base]))
    got = oracle_mod.generate(net(n_nodes, [with_ids(base, f[s0:s0 + ns], f[t0:t0 + nt])]))
    assert ref["src"].size > 0
    np.testing.assert_array_equal(got["src"], f[ref["src"]])
    np.testing.assert_array_equal(got["tgt"], f[ref["tgt"]])
    np.testing.assert_array_equal(got["delay"], ref["delay"])
    np.testing.assert_array_equal(got["weight"], ref["weight"])


@pytest.mark.parametrize("rule", ["one_to_one", "all_to_all", "fixed_indegree", "fixed_outdegree",
                                  "fixed_total_number", "pairwise_bernoulli"])
def test_any_map_commutes_when_autapses_and_multapses_are_allowed(oracle_mod, rule):
    """With both allowed no node comparison is made, so even a map with
    repeated ids commutes (sources and targets of different lengths, so a
    swapped list is caught)."""
    n_nodes = 60
    base = range_proj(rule, True, True, src=(0, 30), tgt=(0, 30 if rule == "one_to_one" else 45))
    rng = np.random.default_rng(8)
    gs = rng.integers(0, n_nodes, base.src[1]).astype(np.uint32)
    gt = rng.integers(0, n_nodes, base.tgt[1]).astype(np.uint32)
    ref = oracle_mod.generate(net(n_nodes, [base]))
    got = oracle_mod.generate(net(n_nodes, [with_ids(base, gs, gt)]))
    np.testing.assert_array_equal(got["src"], gs[ref["src"]])
    np.testing.assert_array_equal(got["tgt"], gt[ref["tgt"]])
    np.testing.assert_array_equal(got["weight"], ref["weight"])


def test_autapse_skip_is_uniform_over_the_other_nodes(oracle_mod):
    """In-degree with autapses off, sources listed out of order and sharing
    some nodes with the targets: no autapse, and every allowed source equally
    likely (chi-square) for each target."""
    src_ids = np.array([17, 3, 11, 8, 5, 14], np.uint32)
    tgt_ids = np.array([8, 2, 17, 5], np.uint32)
    K = 6000
    pj = Projection(src=(0, 6), tgt=(0, 4), rule="fixed_indegree", k=K, autapses=False, multapses=True,
                    src_ids=src_ids, tgt_ids=tgt_ids, **WD)
    g = oracle_mod.generate(net(20, [pj], seed=3))
    assert g["src"].size == 4 * K
    assert not np.any(g["src"] == g["tgt"])
    for t in tgt_ids:
        got = g["src"][g["tgt"] == t]
        allowed = [s for s in src_ids if s != t]
        assert set(got.tolist()) <= set(int(s) for s in allowed)
        counts = np.array([np.sum(got == s) for s in allowed])
        assert stats.chisquare(counts).pvalue > 1e-4


def test_weight_numbers_follow_the_index_formulas(oracle_mod):
    """Weights 0, 1, 2, ... reveal each connection's number i (Sec. 2.1):
    one_to_one i -> (S[i], T[i]); all_to_all i -> (S[i // Nt], T[i mod Nt]);
    in-degree target T[i // K]; out-degree source S[i // K]; fixed total
    number: slot order.  Pairs dropped as autapses leave their number unused."""
    pool = np.random.default_rng(11).permutation(50).astype(np.uint32)
    S = pool[:12]
    T = np.concatenate([pool[12:15], S[5:6], pool[15:20]])  # T[3] = S[5]: one shared node
    for rule, k, ns, nt in (("one_to_one", 0, 9, 9), ("all_to_all", 0, 12, 9), ("fixed_indegree", 5, 12, 9),
                            ("fixed_outdegree", 4, 12, 9), ("fixed_total_number", 50, 12, 9)):
        for aut, mult in FLAGS:
            Si, Ti = S[:ns], T[:nt]
            n_num = {"one_to_one": ns, "all_to_all": ns * nt, "fixed_indegree": nt * k,
                     "fixed_outdegree": ns * k, "fixed_total_number": k}[rule]
            pj = Projection(src=(0, ns), tgt=(0, nt), rule=rule, k=k, autapses=aut, multapses=mult,
                            src_ids=Si, tgt_ids=Ti, weights=np.arange(n_num, dtype=np.float32), **WD)
            g = oracle_mod.generate(net(50, [pj]))
            i = g["weight"].astype(np.int64)
            np.testing.assert_array_equal(i, g["weight"])  # whole numbers
            assert np.all(np.diff(i) > 0), "generation order is the numbering"
            if rule == "one_to_one":
                np.testing.assert_array_equal(g["src"], Si[i])
                np.testing.assert_array_equal(g["tgt"], Ti[i])
                expect = [j for j in range(ns) if aut or Si[j] != Ti[j]]
                np.testing.assert_array_equal(i, expect)
            elif rule == "all_to_all":
                np.testing.assert_array_equal(g["src"], Si[i // nt])
                np.testing.assert_array_equal(g["tgt"], Ti[i % nt])
                expect = [j for j in range(ns * nt) if aut or Si[j // nt] != Ti[j % nt]]
                np.testing.assert_array_equal(i, expect)
            elif rule == "fixed_indegree":
                np.testing.assert_array_equal(g["tgt"], Ti[i // k])
                np.testing.assert_array_equal(i, np.arange(n_num))
            elif rule == "fixed_outdegree":
                np.testing.assert_array_equal(g["src"], Si[i // k])
                np.testing.assert_array_equal(i, np.arange(n_num))
            else:
                np.testing.assert_array_equal(i, np.arange(n_num))
            if not aut:
                assert not np.any(g["src"] == g["tgt"])


def test_per_connection_arrays_leave_the_connectivity_unchanged(oracle_mod):
    """Given weights and delays replace the drawn ones; the endpoints still
    come from the same draws."""
    base = range_proj("fixed_indegree", False, False)
    n = base.tgt[1] * base.k
    rng = np.random.default_rng(2)
    w = rng.normal(0, 1, n).astype(np.float32)
    d = rng.uniform(0.1, 4.0, n).astype(np.float32)
    ref = oracle_mod.generate(net(80, [base]))
    arr = Projection(**{**base.__dict__, "weights": w, "delays": d})
    got = oracle_mod.generate(net(80, [arr]))
    np.testing.assert_array_equal(got["src"], ref["src"])
    np.testing.assert_array_equal(got["tgt"], ref["tgt"])
    np.testing.assert_array_equal(got["weight"], w)


def test_delay_array_steps_hand_computed(oracle_mod):
    """Sec. 2.1: round(d / dt) steps, at least one.  dt = 0.125 ms is binary,
    so every quotient below is exact and the expected steps are read off."""
    d = np.array([0.0, 0.0625, 0.1875, 0.25, 0.3125, -1.0, 8191.875, 1.0, 0.375, 0.4375, 100.0625, 0.125],
                 np.float32)
    #            0 -> 1  .5 -> 1 1.5 -> 2  2 -> 2 2.5 -> 3  <1 -> 1   65535   8        3      3.5 -> 4  800.5 -> 801  1
    expect = [1, 1, 2, 2, 3, 1, 65535, 8, 3, 4, 801, 1]
    n = d.size
    pj = Projection(src=(0, n), tgt=(0, n), rule="one_to_one", src_ids=np.arange(n, dtype=np.uint32),
                    tgt_ids=np.arange(n, 2 * n, dtype=np.uint32), delays=d)
    g = oracle_mod.generate(net(2 * n, [pj], dt=0.125))
    np.testing.assert_array_equal(g["delay"], expect)
    np.testing.assert_array_equal(g["weight"], np.ones(n, np.float32))  # the const distribution stays


def test_equal_delay_array_is_the_constant_delay(oracle_mod):
    base = range_proj("all_to_all", True, True)
    n = base.src[1] * base.tgt[1]
    const = Projection(**{**base.__dict__, "delay": Dist("const", 1.49)})
    arr = Projection(**{**base.__dict__, "delays": np.full(n, 1.49, np.float32)})
    a = oracle_mod.generate(net(80, [const]))
    b = oracle_mod.generate(net(80, [arr]))
    # 1.49 as float32 and as double round to the same step (15)
    np.testing.assert_array_equal(a["delay"], b["delay"])
    assert set(a["delay"].tolist()) == {15}


def test_complete_cases_with_arrays(oracle_mod):
    """K = every candidate (in-degree, no multapses): each target takes all
    of its other sources; N = every allowed pair (total number, neither
    allowed): each allowed pair once."""
    S = np.array([9, 4, 13, 1, 7], np.uint32)
    T = np.array([7, 13, 2, 9], np.uint32)
    pj = Projection(src=(0, 5), tgt=(0, 4), rule="fixed_indegree", k=4, autapses=False, multapses=False,
                    src_ids=S, tgt_ids=T, **WD)
    g = oracle_mod.generate(net(16, [pj]))
    for t in (7, 13, 9):  # sources too: exactly their four other sources
        got = sorted(g["src"][g["tgt"] == t].tolist())
        assert got == sorted(int(s) for s in S if s != t)
    # target 2 is not a source: it has five candidates and takes four distinct ones
    got2 = g["src"][g["tgt"] == 2].tolist()
    assert len(got2) == 4 and len(set(got2)) == 4 and set(got2) <= set(S.tolist())
    allowed = [(int(s), int(t)) for s, t in itertools.product(S, T) if s != t]
    pj = Projection(src=(0, 5), tgt=(0, 4), rule="fixed_total_number", k=len(allowed), autapses=False,
                    multapses=False, src_ids=S, tgt_ids=T, **WD)
    g = oracle_mod.generate(net(16, [pj]))
    assert sorted(zip(g["src"].tolist(), g["tgt"].tolist())) == sorted(allowed)


def test_primary_generation_with_arrays(oracle_mod):
    """generate_primary equals the matching run of generate with arrays."""
    rng = np.random.default_rng(4)
    S = rng.permutation(70)[:30].astype(np.uint32)
    T = rng.permutation(70)[:25].astype(np.uint32)
    n_num = {"fixed_indegree": 25 * 7, "fixed_outdegree": 30 * 7, "all_to_all": 30 * 25}
    for rule, numbered in itertools.product(("fixed_indegree", "fixed_outdegree", "pairwise_bernoulli",
                                             "all_to_all"), (False, True)):
        if numbered and rule not in n_num:
            continue
        extra = dict(weights=np.arange(n_num[rule], dtype=np.float32)) if numbered else {}
        pj = Projection(src=(0, 30), tgt=(0, 25), rule=rule, autapses=False, multapses=False, src_ids=S,
                        tgt_ids=T, **rule_kw(rule), **WD, **extra)
        spec = net(70, [pj])
        g = oracle_mod.generate(spec)
        for b in (0, 7, 24):
            one = oracle_mod.generate_primary(spec, 0, b)
            node = S[b] if rule == "fixed_outdegree" else T[b]
            sel = (g["src"] == node) if rule == "fixed_outdegree" else (g["tgt"] == node)
            for key in ("src", "tgt", "delay", "weight"):
                np.testing.assert_array_equal(one[key], g[key][sel])


def test_build_sorts_array_networks_by_node(oracle_mod):
    S = np.array([30, 2, 17, 9], np.uint32)
    T = np.array([5, 30, 12], np.uint32)
    pj = Projection(src=(0, 4), tgt=(0, 3), rule="all_to_all", src_ids=S, tgt_ids=T, **WD)
    b = oracle_mod.build(net(31, [pj]))
    assert b["src"].size == 12
    assert np.all(np.diff(b["src"].astype(np.int64)) >= 0)
    np.testing.assert_array_equal(np.diff(b["row_ptr"].astype(np.int64))[S], np.full(4, 3))


@pytest.mark.parametrize("case,status", [
    ("id_out_of_range", "INVALID_ARG"),
    ("dup_src_nomult", "INVALID_ARG"),
    ("dup_tgt_nomult", "INVALID_ARG"),
    ("dup_src_noaut_indegree", "INVALID_ARG"),
    ("dup_tgt_noaut_indegree", "OK"),
    ("dup_tgt_noaut_outdegree", "INVALID_ARG"),
    ("dup_src_noaut_all_to_all", "OK"),
    ("k_above_candidates", "INVALID_ARG"),
    ("k_at_candidates", "OK"),
    ("n_above_allowed_pairs", "INVALID_ARG"),
    ("n_at_allowed_pairs", "OK"),
    ("weights_wrong_length", "INVALID_ARG"),
    ("weights_bernoulli", "INVALID_ARG"),
    ("delay_nan", "INVALID_ARG"),
    ("delay_inf", "INVALID_ARG"),
    ("delay_step_65536", "UNSUPPORTED"),
    ("empty_lists", "OK"),
])
def test_array_argument_checks(oracle_mod, case, status):
    S = np.array([3, 8, 1, 6], np.uint32)
    T = np.array([6, 0, 3], np.uint32)  # shares 3 and 6 with S
    kw = dict(src=(0, 4), tgt=(0, 3), rule="fixed_indegree", k=2, autapses=True, multapses=True,
              src_ids=S, tgt_ids=T)
    if case == "id_out_of_range":
        kw["src_ids"] = np.array([3, 8, 1, 10], np.uint32)
    elif case == "dup_src_nomult":
        kw.update(src_ids=np.array([3, 8, 3, 6], np.uint32), multapses=False)
    elif case == "dup_tgt_nomult":
        kw.update(tgt_ids=np.array([6, 0, 6], np.uint32), multapses=False)
    elif case == "dup_src_noaut_indegree":
        kw.update(src_ids=np.array([3, 8, 3, 6], np.uint32), autapses=False)
    elif case == "dup_tgt_noaut_indegree":
        kw.update(tgt_ids=np.array([6, 0, 6], np.uint32), autapses=False)
    elif case == "dup_tgt_noaut_outdegree":
        kw.update(tgt_ids=np.array([6, 0, 6], np.uint32), autapses=False, rule="fixed_outdegree")
    elif case == "dup_src_noaut_all_to_all":
        kw.update(src_ids=np.array([3, 8, 3, 6], np.uint32), autapses=False, rule="all_to_all")
    elif case in ("k_above_candidates", "k_at_candidates"):
        # targets 6 and 3 are sources too: they have 3 candidates
        kw.update(autapses=False, multapses=False, k=4 if case == "k_above_candidates" else 3)
    elif case in ("n_above_allowed_pairs", "n_at_allowed_pairs"):
        kw.update(rule="fixed_total_number", autapses=False, multapses=False,
                  k=4 * 3 - 2 + (1 if case == "n_above_allowed_pairs" else 0))
    elif case == "weights_wrong_length":
        kw["weights"] = np.zeros(5, np.float32)
    elif case == "weights_bernoulli":
        # refused for the rule itself, whatever the array's length
        kw.update(rule="pairwise_bernoulli", p=0.5, k=2, weights=np.zeros(2, np.float32))
    elif case.startswith("delay_"):
        d = np.full(6, 1.0, np.float32)
        d[2] = {"delay_nan": np.nan, "delay_inf": np.inf, "delay_step_65536": 6553.6}[case]
        kw["delays"] = d
    elif case == "empty_lists":
        kw.update(src=(0, 0), tgt=(0, 0), src_ids=np.zeros(0, np.uint32), tgt_ids=np.zeros(0, np.uint32),
                  weights=np.zeros(0, np.float32))
    spec = net(10, [Projection(**kw)])
    assert oracle_mod.STATUS[oracle_mod.check_projection(spec, 0)] == status
    if status == "OK":
        g = oracle_mod.generate(spec)
        if case == "empty_lists":
            assert g["src"].size == 0


def test_marshalling_checks_lengths(oracle_mod):
    pj = Projection(src=(0, 3), tgt=(0, 2), rule="all_to_all", src_ids=np.arange(4, dtype=np.uint32),
                    tgt_ids=np.arange(2, dtype=np.uint32))
    with pytest.raises(ValueError):
        oracle_mod.generate(net(10, [pj]))

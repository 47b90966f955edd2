"""Pins of the oracle's connection rules (Sec. 2.1 formulas; Sec. 4 for
pairwise Bernoulli and the autapse / multapse prohibitions).

Deterministic rules are checked by brute-force enumeration and by the
paper's Fig. 1 worked example; random rules by exact counts, prohibitions
and distribution tests (the paper itself checks random connectivity only
statistically, Sec. 2.7).
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import stats

from paper_2306_09855_gb300.workloads import Dist, NetworkSpec, Projection

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
WD = dict(weight=Dist("normal", 1.0, 0.1), delay=Dist("normal", 1.5, 0.75))


def net(pops, projs, seed=1234, dt=0.1):
    return NetworkSpec(seed=seed, dt=dt, populations=list(pops), projections=list(projs))


def pairs(g):
    return list(zip(g["src"].tolist(), g["tgt"].tolist()))


def test_fig1_all_to_all_worked_example(oracle_mod):
    rows = np.loadtxt(os.path.join(GOLDEN, "fig1_all_to_all.txt"), dtype=np.int64)
    spec = net([4, 3], [Projection(src=(0, 4), tgt=(4, 3), rule="all_to_all", **WD)])
    g = oracle_mod.generate(spec)
    assert g["src"].size == 12
    np.testing.assert_array_equal(g["src"], rows[:, 1])
    np.testing.assert_array_equal(g["tgt"] - 4, rows[:, 2])


@pytest.mark.parametrize("s0,t0,n,aut", [(0, 5, 5, True), (0, 5, 5, False), (2, 2, 6, True),
                                         (2, 2, 6, False), (0, 3, 6, False)])
def test_one_to_one_enumeration(oracle_mod, s0, t0, n, aut):
    spec = net([12], [Projection(src=(s0, n), tgt=(t0, n), rule="one_to_one", autapses=aut, **WD)])
    g = oracle_mod.generate(spec)
    expect = [(s0 + i, t0 + i) for i in range(n) if aut or s0 + i != t0 + i]
    assert pairs(g) == expect


@pytest.mark.parametrize("aut", [True, False])
def test_all_to_all_enumeration_overlapping(oracle_mod, aut):
    spec = net([9], [Projection(src=(1, 5), tgt=(3, 6), rule="all_to_all", autapses=aut, **WD)])
    g = oracle_mod.generate(spec)
    expect = [(s, t) for s in range(1, 6) for t in range(3, 9) if aut or s != t]
    assert pairs(g) == expect


def test_rule_counts_and_degrees(oracle_mod):
    spec = net([300, 200], [
        Projection(src=(0, 300), tgt=(300, 200), rule="fixed_indegree", k=17, **WD),
        Projection(src=(300, 200), tgt=(0, 300), rule="fixed_outdegree", k=23, **WD),
        Projection(src=(0, 500), tgt=(0, 500), rule="fixed_total_number", k=12345, **WD),
        Projection(src=(0, 300), tgt=(0, 300), rule="fixed_indegree", k=9, autapses=False,
                   multapses=False, **WD),
    ])
    g = oracle_mod.generate(spec)
    np.testing.assert_array_equal(g["per_proj"], [200 * 17, 200 * 23, 12345, 300 * 9])
    o = np.cumsum(np.concatenate([[0], g["per_proj"]]))
    s, t = g["src"].astype(np.int64), g["tgt"].astype(np.int64)
    # indegree: each target exactly K, sources in range, target-major order
    sl = slice(o[0], o[1])
    assert np.all(np.bincount(t[sl] - 300, minlength=200) == 17)
    assert np.all(np.diff(t[sl]) >= 0) and s[sl].max() < 300
    # outdegree: each source exactly K, source-major order
    sl = slice(o[1], o[2])
    assert np.all(np.bincount(s[sl] - 300, minlength=200) == 23)
    assert np.all(np.diff(s[sl]) >= 0) and t[sl].max() < 300
    # total number: everything in range
    sl = slice(o[2], o[3])
    assert s[sl].max() < 500 and t[sl].max() < 500
    # no autapse, no multapse
    sl = slice(o[3], o[4])
    assert np.all(s[sl] != t[sl])
    assert len(set(zip(s[sl], t[sl]))) == 300 * 9


def test_indegree_sources_uniform(oracle_mod):
    spec = net([50, 4000], [Projection(src=(0, 50), tgt=(50, 4000), rule="fixed_indegree", k=25, **WD)])
    g = oracle_mod.generate(spec)
    h = np.bincount(g["src"], minlength=50)
    assert stats.chisquare(h).pvalue > 1e-4


def test_outdegree_targets_uniform_without_autapses(oracle_mod):
    spec = net([40], [Projection(src=(0, 40), tgt=(0, 40), rule="fixed_outdegree", k=500,
                                 autapses=False, **WD)])
    g = oracle_mod.generate(spec)
    s, t = g["src"].astype(np.int64), g["tgt"].astype(np.int64)
    assert np.all(s != t)
    # per source: the 39 other nodes equally likely
    counts = np.zeros((40, 40), np.int64)
    np.add.at(counts, (s, t), 1)
    off = counts[~np.eye(40, dtype=bool)].reshape(40, 39)
    for row in off[:5]:
        assert stats.chisquare(row).pvalue > 1e-5
    assert stats.chisquare(off.sum(axis=0)).pvalue > 1e-4


@pytest.mark.parametrize("k,aut", [(2, True), (4, True), (2, False), (3, False)])
def test_no_multapse_subsets_equally_likely(oracle_mod, k, aut):
    """Every k-subset of the candidates is equally frequent; k > half of the
    candidates exercises the complement selection."""
    n_src, n_tgt = 5, 6000
    first_t = 0 if not aut else 5
    pops = [n_src + n_tgt] if not aut else [n_src, n_tgt]
    spec = net(pops, [Projection(src=(0, n_src), tgt=(first_t, n_tgt), rule="fixed_indegree", k=k,
                                 autapses=aut, multapses=False, **WD)])
    g = oracle_mod.generate(spec)
    s = g["src"].reshape(n_tgt, k).astype(np.int64)
    tg = g["tgt"].reshape(n_tgt, k)[:, 0].astype(np.int64)
    rows = [tuple(sorted(r)) for r in s]
    assert all(len(set(r)) == k for r in rows)
    # use targets whose candidate set is the full source range (no self in range)
    full = [r for r, t in zip(rows, tg) if t >= n_src or aut]
    cnt = {c: 0 for c in itertools.combinations(range(n_src), k)}
    for r in full:
        cnt[r] += 1
    assert stats.chisquare(list(cnt.values())).pvalue > 1e-4
    if not aut:
        for r, t in zip(rows, tg):
            assert t not in r


def test_no_multapse_slot_order_is_uniform_permutation(oracle_mod):
    """In the first-distinct mode the ordered K-tuple is uniform over the
    K-permutations (draws are exchangeable)."""
    spec = net([4, 8000], [Projection(src=(0, 4), tgt=(4, 8000), rule="fixed_indegree", k=2,
                                      multapses=False, **WD)])
    g = oracle_mod.generate(spec)
    s = g["src"].reshape(-1, 2)
    codes = s[:, 0].astype(np.int64) * 4 + s[:, 1]
    h = np.bincount(codes, minlength=16)
    h = h[[a * 4 + b for a in range(4) for b in range(4) if a != b]]
    assert stats.chisquare(h).pvalue > 1e-4


def test_complement_mode_lists_ascending(oracle_mod):
    spec = net([10, 50], [Projection(src=(0, 10), tgt=(10, 50), rule="fixed_indegree", k=8,
                                     multapses=False, **WD)])
    g = oracle_mod.generate(spec)
    s = g["src"].reshape(50, 8)
    assert np.all(np.diff(s.astype(np.int64), axis=1) > 0)


@pytest.mark.parametrize("aut,mult", [(True, True), (False, True), (True, False), (False, False)])
def test_total_number_prohibitions(oracle_mod, aut, mult):
    spec = net([6], [Projection(src=(0, 6), tgt=(0, 6), rule="fixed_total_number",
                                k=30 if not mult else 200, autapses=aut, multapses=mult, **WD)])
    g = oracle_mod.generate(spec)
    p = pairs(g)
    assert len(p) == (30 if not mult else 200)
    if not aut:
        assert all(s != t for s, t in p)
    if not mult:
        assert len(set(p)) == len(p)


def test_total_number_no_multapse_uniform_subsets(oracle_mod):
    """Fill 5 of the 6 allowed pairs of a 2x3 block: each left-out pair is
    equally likely over seeds (the accepted set is a uniform subset)."""
    miss = []
    for seed in range(1500):
        spec = net([5], [Projection(src=(0, 2), tgt=(2, 3), rule="fixed_total_number", k=5,
                                    multapses=False, **WD)], seed=seed)
        g = oracle_mod.generate(spec)
        allp = {(s, t) for s in range(2) for t in range(2, 5)}
        left = allp - set(pairs(g))
        assert len(left) == 1
        miss.append(sorted(allp).index(left.pop()))
    assert stats.chisquare(np.bincount(miss, minlength=6)).pvalue > 1e-4


def test_total_number_pair_uniformity(oracle_mod):
    spec = net([7, 9], [Projection(src=(0, 7), tgt=(7, 9), rule="fixed_total_number", k=60000, **WD)])
    g = oracle_mod.generate(spec)
    codes = g["src"].astype(np.int64) * 9 + (g["tgt"].astype(np.int64) - 7)
    assert stats.chisquare(np.bincount(codes, minlength=63)).pvalue > 1e-4


@pytest.mark.parametrize("aut", [True, False])
def test_bernoulli_counts_binomial(oracle_mod, aut):
    n_src, n_tgt, p = 400, 3000, 0.05
    pops = [n_src, n_tgt] if aut else [n_tgt]
    tfirst = n_src if aut else 0
    spec = net(pops, [Projection(src=(0, n_src), tgt=(tfirst, n_tgt), rule="pairwise_bernoulli",
                                 p=p, autapses=aut, **WD)])
    g = oracle_mod.generate(spec)
    t = g["tgt"].astype(np.int64) - tfirst
    s = g["src"].astype(np.int64)
    cnt = np.bincount(t, minlength=n_tgt)
    if not aut:
        assert np.all(s != g["tgt"].astype(np.int64))
        cand = np.where(np.arange(n_tgt) < n_src, n_src - 1, n_src)
    else:
        cand = np.full(n_tgt, n_src)
    # no duplicate pair
    assert np.unique(s * 10**6 + t).size == s.size
    # per-target counts follow Binomial(candidates, p): probability-integral check
    sel = cand == n_src
    c = cnt[sel]
    edges = np.arange(0, 50)
    obs = np.bincount(np.minimum(c, 49), minlength=50)
    prob = stats.binom.pmf(edges, n_src, p)
    prob[-1] = stats.binom.sf(48, n_src, p)
    exp = prob * c.size
    keep = exp > 5
    chi2 = np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep]) + 0.0
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4
    # marginal probability of each candidate source ~ p
    hs = np.bincount(s[sel[t]], minlength=n_src)
    assert abs(hs.mean() / sel.sum() - p) < 0.002


def test_bernoulli_extremes(oracle_mod):
    spec = net([4, 5], [Projection(src=(0, 4), tgt=(4, 5), rule="pairwise_bernoulli", p=1.0, **WD),
                        Projection(src=(0, 4), tgt=(4, 5), rule="pairwise_bernoulli", p=0.0, **WD)])
    g = oracle_mod.generate(spec)
    np.testing.assert_array_equal(g["per_proj"], [20, 0])
    assert sorted(pairs(g)) == sorted((s, t) for s in range(4) for t in range(4, 9))


@pytest.mark.parametrize("proj,status", [
    (Projection(src=(0, 3), tgt=(3, 4), rule="one_to_one", **WD), "INVALID_ARG"),
    (Projection(src=(0, 3), tgt=(3, 4), rule="fixed_indegree", k=4, multapses=False, **WD), "INVALID_ARG"),
    (Projection(src=(0, 3), tgt=(0, 3), rule="fixed_indegree", k=3, autapses=False, multapses=False, **WD),
     "INVALID_ARG"),
    (Projection(src=(0, 3), tgt=(3, 4), rule="fixed_indegree", k=3, multapses=False, **WD), None),
    (Projection(src=(0, 1), tgt=(0, 1), rule="fixed_total_number", k=1, autapses=False, **WD),
     "INVALID_ARG"),
    (Projection(src=(0, 2), tgt=(2, 2), rule="fixed_total_number", k=5, multapses=False, **WD),
     "INVALID_ARG"),
    (Projection(src=(0, 3), tgt=(5, 4), rule="all_to_all", **WD), "INVALID_ARG"),
    (Projection(src=(0, 3), tgt=(3, 4), rule="pairwise_bernoulli", p=1.5, **WD), "INVALID_ARG"),
])
def test_connect_validation(oracle_mod, proj, status):
    spec = net([3, 4], [proj])
    st = oracle_mod.check_projection(spec, 0)
    if status is None:
        assert st == 0
    else:
        assert oracle_mod.STATUS[st] == status


def test_deterministic_and_seed_sensitive(oracle_mod):
    mk = lambda seed: net([200], [Projection(src=(0, 200), tgt=(0, 200), rule="fixed_indegree", k=10,
                                             **WD)], seed=seed)
    a, b, c = oracle_mod.generate(mk(5)), oracle_mod.generate(mk(5)), oracle_mod.generate(mk(6))
    for key in ("src", "tgt", "delay", "weight"):
        np.testing.assert_array_equal(a[key], b[key])
    assert np.mean(a["src"] == c["src"]) < 0.05


@pytest.mark.parametrize("rule,extra", [("fixed_indegree", dict(k=7)), ("fixed_outdegree", dict(k=5)),
                                        ("pairwise_bernoulli", dict(p=0.1)), ("all_to_all", {}),
                                        ("one_to_one", {}),
                                        ("fixed_indegree", dict(k=30, multapses=False, autapses=False))])
def test_generate_primary_matches_full_generation(oracle_mod, rule, extra):
    spec = net([40], [Projection(src=(0, 40), tgt=(0, 40), rule=rule, **extra, **WD)])
    g = oracle_mod.generate(spec)
    if rule == "all_to_all":
        # full generation is source-major; per-target view lists sources ascending
        for b in (0, 17, 39):
            one = oracle_mod.generate_primary(spec, 0, b)
            sel = g["tgt"] == b
            np.testing.assert_array_equal(one["src"], g["src"][sel])
            np.testing.assert_array_equal(one["weight"], g["weight"][sel])
        return
    key = "src" if rule == "fixed_outdegree" else "tgt"
    for b in (0, 17, 39):
        one = oracle_mod.generate_primary(spec, 0, b)
        sel = np.nonzero(g[key] == b)[0]
        if rule == "one_to_one":
            sel = sel[:1]
        for f in ("src", "tgt", "delay", "weight"):
            np.testing.assert_array_equal(one[f], g[f][sel])

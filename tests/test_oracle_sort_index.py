"""Pins of the oracle's sort and group index (Sec. 2.2).

Connections are ordered by source, then delay (the paper's two sort keys),
ties in generation order (a stable sort); a connection starts a group when its
source or delay differs from its predecessor; G_i is the number of groups of
source i and p_i = sum_{j<i} G_j with p_0 = 0.
Checked against numpy's stable lexsort, bincount and a per-source count of
distinct delays.
"""
import numpy as np
import pytest

from paper_2306_09855_gb300 import workloads as W
from paper_2306_09855_gb300.workloads import Dist, NetworkSpec, Projection


def _specs():
    yield W.plain_indegree(n=300, k=20)
    yield W.two_population(200, "fixed_total_number", k=30000)
    yield W.two_population(150, "pairwise_bernoulli", p=0.05, autapses=False)
    yield NetworkSpec(seed=9, dt=1.0, populations=[30], projections=[
        Projection(src=(0, 30), tgt=(0, 30), rule="fixed_total_number", k=5000,
                   weight=Dist("normal", 0.0, 1.0), delay=Dist("const", 2.0))])


@pytest.mark.parametrize("spec", list(_specs()), ids=lambda s: s.name or "const_delay")
def test_sort_and_index_against_numpy(oracle_mod, spec):
    g = oracle_mod.generate(spec)
    o = oracle_mod.sort_index(spec.n_nodes, g["src"], g["tgt"], g["delay"], g["weight"])
    order = np.lexsort((np.arange(g["src"].size), g["delay"], g["src"]))
    for f in ("src", "tgt", "delay", "weight"):
        np.testing.assert_array_equal(o[f], g[f][order])
    n_nodes = spec.n_nodes
    deg = np.bincount(g["src"], minlength=n_nodes)
    np.testing.assert_array_equal(o["row_ptr"], np.concatenate([[0], np.cumsum(deg)]))
    s = o["src"].astype(np.int64)
    d = o["delay"].astype(np.int64)
    starts = np.nonzero(np.concatenate([[True], (np.diff(s) != 0) | (np.diff(d) != 0)]))[0]
    np.testing.assert_array_equal(o["group_first"], starts)
    pairs = np.unique(g["src"].astype(np.int64) * 65536 + g["delay"])
    G = np.bincount(pairs // 65536, minlength=n_nodes)
    np.testing.assert_array_equal(o["group_ptr"], np.concatenate([[0], np.cumsum(G)]))
    assert o["n_groups"] == pairs.size


def test_empty_network(oracle_mod):
    o = oracle_mod.sort_index(5, [], [], [], [])
    assert o["n_groups"] == 0
    np.testing.assert_array_equal(o["row_ptr"], np.zeros(6))

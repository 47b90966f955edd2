"""Pins of the oracle's spike delivery (Sec. 2.3): every group of every
source delivered once gives the column sums of the weight matrix; one group
touches exactly the source's connections of that delay; the input is linear
in the multiplicity; and a hand-computed example."""
import numpy as np
import pytest

from paper_2306_09855_gb300.workloads import Dist, NetworkSpec, Projection


@pytest.fixture(scope="module")
def net(oracle_mod):
    spec = NetworkSpec(seed=7, dt=0.1, populations=[300, 200], projections=[
        Projection(src=(0, 300), tgt=(300, 200), rule="fixed_indegree", k=30,
                   weight=Dist("normal", 5.0, 1.0), delay=Dist("normal", 1.5, 0.75)),
        Projection(src=(300, 200), tgt=(0, 500), rule="pairwise_bernoulli", p=0.05,
                   weight=Dist("normal", -20.0, 2.0), delay=Dist("normal", 0.75, 0.375))])
    return spec, oracle_mod.build(spec)


def _all_groups(out):
    gp = out["group_ptr"].astype(np.int64)
    g = np.diff(gp)
    src = np.repeat(np.arange(g.size, dtype=np.uint32), g)
    grp = np.concatenate([np.arange(k, dtype=np.uint32) for k in g]) if g.sum() else np.zeros(0, np.uint32)
    return src, grp


def test_every_group_once_gives_column_sums(oracle_mod, net):
    spec, out = net
    src, grp = _all_groups(out)
    r = oracle_mod.deliver(out, spec.n_nodes, src, grp, np.ones(src.size, np.float32))
    expect = np.bincount(out["tgt"].astype(np.int64), weights=out["weight"].astype(np.float64),
                         minlength=spec.n_nodes)
    np.testing.assert_allclose(r["input"], expect, rtol=1e-12, atol=1e-9)
    assert r["bad"] == 0
    np.testing.assert_array_equal(r["terms"], np.bincount(out["tgt"].astype(np.int64), minlength=spec.n_nodes))


def test_one_group_is_one_source_and_delay(oracle_mod, net):
    spec, out = net
    rng = np.random.default_rng(3)
    row = np.diff(out["row_ptr"].astype(np.int64))
    s_of = np.repeat(np.arange(spec.n_nodes), row)
    for s in rng.choice(np.flatnonzero(row > 0), 20, replace=False):
        delays = np.unique(out["delay"][s_of == s])
        for k in (0, delays.size - 1, delays.size // 2):
            m = np.float32(rng.uniform(0.5, 3.0))
            r = oracle_mod.deliver(out, spec.n_nodes, [s], [k], [m])
            sel = (s_of == s) & (out["delay"] == delays[k])
            expect = np.bincount(out["tgt"][sel].astype(np.int64),
                                 weights=out["weight"][sel].astype(np.float64) * float(m), minlength=spec.n_nodes)
            np.testing.assert_allclose(r["input"], expect, rtol=1e-12, atol=1e-9)


def test_linear_in_multiplicity_and_bad_entries(oracle_mod, net):
    spec, out = net
    src, grp = _all_groups(out)
    a = oracle_mod.deliver(out, spec.n_nodes, src, grp, np.full(src.size, 1.0, np.float32))
    b = oracle_mod.deliver(out, spec.n_nodes, src, grp, np.full(src.size, 3.0, np.float32))
    np.testing.assert_allclose(b["input"], 3.0 * a["input"], rtol=1e-12, atol=1e-9)
    n_groups = np.diff(out["group_ptr"].astype(np.int64))
    c = oracle_mod.deliver(out, spec.n_nodes, [spec.n_nodes, 0, 1], [0, int(n_groups[0]), 0], [1.0, 1.0, 1.0])
    assert c["bad"] == 2


def test_hand_example(oracle_mod):
    # Source 0: (t=1, d=1, w=1.5), (t=2, d=1, w=-2), (t=2, d=3, w=0.25);
    # source 1: none; source 2: (t=0, d=2, w=4).  Groups: [0, 2) and [2, 3)
    # of source 0, [3, 4) of source 2.
    out = {"row_ptr": np.array([0, 3, 3, 4], np.uint64), "group_ptr": np.array([0, 2, 2, 3], np.uint64),
           "group_first": np.array([0, 2, 3], np.uint64), "tgt": np.array([1, 2, 2, 0], np.uint32),
           "weight": np.array([1.5, -2.0, 0.25, 4.0], np.float32)}
    r = oracle_mod.deliver(out, 3, [0, 0, 2, 1, 0], [0, 1, 0, 0, 2], [1.0, 2.0, 0.5, 1.0, 1.0])
    np.testing.assert_array_equal(r["input"], [2.0, 1.5, -1.5])
    np.testing.assert_array_equal(r["terms"], [1, 1, 2])
    np.testing.assert_array_equal(r["abs"], [2.0, 1.5, 2.5])
    assert r["bad"] == 2

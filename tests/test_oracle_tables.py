"""Pins of the oracle's delay and binomial threshold tables and its weights.

Delay (Sec. 2.1, last paragraph): the delay in ms is divided by dt, rounded
to an integer and raised to at least one step.  For d ~ N(mu, sigma) this
gives P(step <= k) = Phi(((k + 1/2) dt - mu) / sigma) for k >= 1; the table
holds floor(2^32 P(step <= k)).
Bernoulli count (pairwise Bernoulli, Sec. 4): Binomial(candidates, p).
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2306_09855_gb300 import workloads as W


def _table_value(base, thr, u):
    return base + np.searchsorted(thr, u, side="right")


@pytest.mark.parametrize("mu,sigma,dt", [(1.5, 0.75, 0.1), (0.75, 0.375, 0.1), (5.0, 0.01, 0.1),
                                         (0.02, 0.05, 0.1), (30.0, 4.0, 0.25), (1.0, 2.0, 1.0)])
def test_delay_table_matches_normal_cdf(oracle_mod, mu, sigma, dt):
    base, thr = oracle_mod.delay_table(mu, sigma, dt)
    assert base >= 1
    assert np.all(np.diff(thr.astype(np.int64)) >= 0)
    ks = np.arange(base, base + thr.size)
    cdf = stats.norm.cdf(((ks + 0.5) * dt - mu) / sigma)
    expect = np.floor(cdf * 2.0 ** 32)
    assert np.max(np.abs(expect - thr.astype(np.float64))) <= 2.0
    # below the base: probability below one part in 2^32; after the table: above 1 - 2^-32
    if base > 1:
        assert stats.norm.cdf(((base - 1 + 0.5) * dt - mu) / sigma) < 2.0 ** -32 * 2
    top = base + thr.size
    assert stats.norm.cdf(((top + 0.5) * dt - mu) / sigma) > 1 - 2.0 ** -31


def test_delay_rounding_rule_against_sampled_normals(oracle_mod):
    """Steps from the table follow the law of max(1, round(d/dt)) of normal samples."""
    mu, sigma, dt = 1.5, 0.75, 0.1
    base, thr = oracle_mod.delay_table(mu, sigma, dt)
    rng = np.random.default_rng(7)
    n = 400_000
    u = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    steps_table = _table_value(base, thr, u)
    d = rng.normal(mu, sigma, n)
    steps_direct = np.maximum(1, np.floor(d / dt + 0.5)).astype(np.int64)
    hi = 40
    a = np.bincount(np.minimum(steps_table, hi), minlength=hi + 1)[1:]
    b = np.bincount(np.minimum(steps_direct, hi), minlength=hi + 1)[1:]
    keep = (a + b) > 20
    chi2, pval, _, _ = stats.chi2_contingency(np.stack([a[keep], b[keep]]))
    assert pval > 1e-4, pval


def test_delay_steps_of_generated_network(oracle_mod):
    """Delays the oracle draws for a whole network: chi-square against Phi."""
    spec = W.plain_indegree(n=1000, k=100)
    g = oracle_mod.generate(spec)
    steps = g["delay"].astype(np.int64)
    assert steps.min() >= 1
    dt, mu, sigma = 0.1, 1.5, 0.75
    kmax = 40
    obs = np.bincount(np.minimum(steps, kmax), minlength=kmax + 1)[1:]
    edges = np.arange(1, kmax + 1)
    upper = stats.norm.cdf(((edges + 0.5) * dt - mu) / sigma)
    lower = np.concatenate([[0.0], upper[:-1]])
    prob = upper - lower
    prob[-1] = 1.0 - lower[-1]
    exp = prob * steps.size
    keep = exp > 5
    chi2 = np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep])
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4


@pytest.mark.parametrize("n,p", [(1000, 0.1), (100_000, 0.01), (99_999, 0.01), (50, 0.5),
                                 (7, 0.999), (20_000, 0.005), (3, 0.3), (1, 0.4)])
def test_binomial_table_matches_scipy(oracle_mod, n, p):
    base, thr = oracle_mod.binom_table(n, p)
    ks = np.arange(base, base + thr.size)
    expect = np.floor(stats.binom.cdf(ks, n, p) * 2.0 ** 32)
    assert np.max(np.abs(expect - thr.astype(np.float64)), initial=0) <= 2.0
    if base > 0:
        assert stats.binom.cdf(base - 1, n, p) < 2.0 ** -31
    assert stats.binom.cdf(base + thr.size, n, p) > 1 - 2.0 ** -31


def test_binomial_table_degenerate(oracle_mod):
    assert oracle_mod.binom_table(0, 0.3) == (0, pytest.approx(np.zeros(0)))
    b, t = oracle_mod.binom_table(10, 0.0)
    assert b == 0 and t.size == 0
    b, t = oracle_mod.binom_table(10, 1.0)
    assert b == 10 and t.size == 0


def test_normal_weight_closed_forms(oracle_mod):
    mu, sigma = 50.0, 5.0
    # u1 = 1 (top 24 bits all ones) -> radius 0 -> w = mu exactly
    assert oracle_mod.normal_weight(mu, sigma, 0xFFFFFF00, 0x12345600) == np.float32(mu)
    # u2 = 0 -> cos = 1 ; u2 = 1/2 -> cos = -1
    for w2 in (0, 0x00ABCD00, 0x7F000000, 0xF0000000):
        u1 = ((w2 >> 8) + 1) * 2.0 ** -24
        r = math.sqrt(-2.0 * math.log(u1))
        assert oracle_mod.normal_weight(mu, sigma, w2, 0) == np.float32(mu + sigma * r)
        assert oracle_mod.normal_weight(mu, sigma, w2, 0x80000000) == np.float32(mu - sigma * r)
        # u2 = 1/4 and 3/4: cos = 0 -> mu
        assert abs(oracle_mod.normal_weight(mu, sigma, w2, 0x40000000) - mu) < 1e-4
    # the low 8 bits of either word are unused
    assert oracle_mod.normal_weight(mu, sigma, 0x12345678, 0x9ABCDEF0) == \
        oracle_mod.normal_weight(mu, sigma, 0x123456FF, 0x9ABCDE00)


def test_normal_weight_distribution(oracle_mod):
    rng = np.random.default_rng(11)
    n = 200_000
    w2 = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    w3 = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    w = oracle_mod.normal_weights(-250.0, 25.0, w2, w3).astype(np.float64)
    assert abs(w.mean() + 250.0) < 4 * 25.0 / math.sqrt(n)
    assert abs(w.std() - 25.0) < 0.01 * 25.0
    assert stats.kstest((w + 250.0) / 25.0, "norm").pvalue > 1e-4


def test_weights_of_generated_network(oracle_mod):
    spec = W.plain_indegree(n=1000, k=100)
    g = oracle_mod.generate(spec)
    exc = g["src"] < 1000
    we = g["weight"][exc].astype(np.float64)
    wi = g["weight"][~exc].astype(np.float64)
    assert stats.kstest((we - 50.0) / 5.0, "norm").pvalue > 1e-4
    assert stats.kstest((wi + 250.0) / 25.0, "norm").pvalue > 1e-4

"""The autotuner's cache key (host logic, no GPU): the expected connection
count of every rule (Sec. 2.1 counts; pairwise_bernoulli its mean) against
the oracle's counts, and the size classes."""
import numpy as np

from paper_2306_09855_gb300 import autotune
from paper_2306_09855_gb300 import workloads as W


def test_expected_counts_match_the_oracle(oracle_mod):
    for rule, mult in W.RULE_SWEEP_RUNS:
        spec = W.rule_sweep(rule, mult, scale=0.01)
        est = autotune._connections([spec])
        n, _ = oracle_mod.count(spec)
        if rule == "pairwise_bernoulli":
            assert abs(n - est) <= 5 * np.sqrt(est) + 1, (rule, n, est)  # binomial spread
        elif (rule in ("one_to_one", "all_to_all")) and not mult:
            assert n <= est  # autapses dropped
        else:
            assert n == est, (rule, mult, n, est)


def test_size_classes():
    assert autotune._size_class(0) == "tiny"
    assert autotune._size_class(999_999) == "tiny"
    assert autotune._size_class(1_000_000) == "small"
    assert autotune._size_class(4 * 10**8) == "large"
    assert autotune._connections([W.microcircuit()]) == 299_999_997  # rint per call: 3e8 - 3
    assert autotune._size_class(autotune._connections([W.rule_sweep("fixed_indegree", True)])) == "large"
    assert autotune._size_class(autotune._connections(W.batched_sweep())) == "large"

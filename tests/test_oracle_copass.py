"""Pins of the oracle's COPASS partition and block sort (Appendix A).

The partition of k sorted runs with left size m must put, in the left
partitions, exactly the first m elements of the stable order of the
concatenated runs (equal keys: lower run first, then position); brute force
on small random runs with many ties checks that, and its defining
properties (sum = m, every left element <= every right element).  The block
sort must equal numpy's stable argsort for any block size.  Planted
mistakes (ties given to the higher run, a partition off by one) fail."""
import numpy as np
import pytest


def _stable_first_m(runs, m):
    keys = np.concatenate([np.asarray(r, np.uint64) for r in runs]) if runs else np.zeros(0, np.uint64)
    run_id = np.concatenate([np.full(len(r), i) for i, r in enumerate(runs)]) if runs else np.zeros(0, int)
    order = np.argsort(keys, kind="stable")[:m]
    return np.bincount(run_id[order], minlength=len(runs))


@pytest.mark.parametrize("seed", range(40))
def test_partition_is_the_first_m_of_the_stable_order(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(1, 7))
    hi = int(rng.choice([3, 10, 1000, 2**40]))  # few distinct values: many ties
    runs = [np.sort(rng.integers(0, hi, int(rng.integers(0, 40)), dtype=np.uint64)) for _ in range(k)]
    total = sum(len(r) for r in runs)
    for m in sorted({0, total, *rng.integers(0, total + 1, 6).tolist()}):
        part = oracle_mod.copass_partition(runs, m)
        assert part.sum() == m
        assert all(0 <= p <= len(r) for p, r in zip(part, runs))
        left = [r[:p] for r, p in zip(runs, part)]
        right = [r[p:] for r, p in zip(runs, part)]
        lmax = max((int(x.max()) for x in left if x.size), default=None)
        rmin = min((int(x.min()) for x in right if x.size), default=None)
        if lmax is not None and rmin is not None:
            assert lmax <= rmin
        np.testing.assert_array_equal(part, _stable_first_m(runs, m))


def test_partition_reaches_both_last_steps(oracle_mod):
    """Distinct keys end in the one-wide intervals (last step, case 1);
    a run of equal keys straddling m ends at a trial threshold equal to the
    answer (last step, case 2)."""
    runs = [np.array([1, 4, 9], np.uint64), np.array([2, 3, 10], np.uint64), np.array([5, 6, 7, 8], np.uint64)]
    for m in range(0, 11):
        np.testing.assert_array_equal(oracle_mod.copass_partition(runs, m), _stable_first_m(runs, m))
    runs = [np.array([1, 5, 5, 5], np.uint64), np.array([5, 5, 6], np.uint64), np.array([0, 5, 9], np.uint64)]
    for m in range(0, 11):
        np.testing.assert_array_equal(oracle_mod.copass_partition(runs, m), _stable_first_m(runs, m))


@pytest.mark.parametrize("n,block,hi", [(1000, 100, 50), (1000, 333, 7), (4097, 512, 2**30), (10, 64, 3),
                                        (777, 1, 5), (2048, 1024, 2**63)])
def test_block_sort_equals_stable_sort(oracle_mod, n, block, hi):
    rng = np.random.default_rng(n + block)
    keys = rng.integers(0, hi, n, dtype=np.uint64)
    vals = np.arange(n, dtype=np.uint64) * np.uint64(3) + np.uint64(7)  # distinct: order visible
    order = np.argsort(keys, kind="stable")
    k, v = oracle_mod.copass_sort(keys, vals, block)
    np.testing.assert_array_equal(k, keys[order])
    np.testing.assert_array_equal(v, vals[order])


def test_block_sort_rejects_zero_block(oracle_mod):
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.copass_sort(np.zeros(3, np.uint64), np.zeros(3, np.uint64), 0)

"""COPASS block sort (Appendix A) on the GPU.

The stand-alone sort (snc_block_sort_pairs) must give numpy's stable order,
and the oracle's COPASS, bit for bit, for ragged last blocks, one block, up
to the 256-block limit, 64-bit keys and heavy ties.  A network built with
the block sort (snc_set_block_sort) must equal the oracle's network; under a
device-memory budget that the out-of-place sort exceeds, the default build
runs out of memory and the block-sorted build succeeds with the same
result."""
import ctypes

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


def _block_sort(snc, keys, vals, bits, block):
    import torch
    k = torch.from_numpy(keys.view(np.int64)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    snc.snc_block_sort_pairs(k.data_ptr(), v.data_ptr(), keys.size, bits, block,
                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return k.cpu().numpy().view(np.uint64), v.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n,block,bits,hi", [
    (100_000, 8192, 25, 1 << 25),      # 13 blocks, ragged last one
    (100_000, 1024, 12, 1 << 6),       # 98 blocks, few distinct keys
    (50_000, 65536, 30, 1 << 30),      # one block
    (262_144, 1024, 20, 1 << 20),      # 256 blocks, the limit
    (300_001, 16384, 64, 1 << 63),     # 64-bit keys
    (200_000, 4096, 17, 3),            # almost all keys equal
])
def test_block_sort_is_the_stable_sort(snc, n, block, bits, hi):
    rng = np.random.default_rng(n + block)
    keys = rng.integers(0, hi, n, dtype=np.uint64)
    if bits == 64:
        keys |= rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)
    vals = np.arange(n, dtype=np.uint32)  # distinct: the order of equal keys is visible
    order = np.argsort(keys, kind="stable")
    k, v = _block_sort(snc, keys, vals, bits, block)
    np.testing.assert_array_equal(k, keys[order])
    np.testing.assert_array_equal(v, vals[order])


def test_block_sort_equals_oracle_copass(snc, oracle_mod):
    rng = np.random.default_rng(4)
    keys = rng.integers(0, 1000, 70_000, dtype=np.uint64)
    vals = rng.integers(0, 1 << 32, 70_000, dtype=np.uint64).astype(np.uint32)
    ok, ov = oracle_mod.copass_sort(keys, vals.astype(np.uint64), 8192)
    k, v = _block_sort(snc, keys, vals, 10, 8192)
    np.testing.assert_array_equal(k, ok)
    np.testing.assert_array_equal(v, ov.astype(np.uint32))


CASES = [("indegree", W.rule_sweep("fixed_indegree", True, scale=0.05), 1 << 21),              # 2e7, 10 blocks
         ("total_nomult", W.rule_sweep("fixed_total_number", False, scale=0.05), 1 << 17),   # 1e6, 8 blocks
         ("bernoulli", W.rule_sweep("pairwise_bernoulli", False, scale=0.05), 1 << 17),      # 1e6, 8 blocks
         ("outdegree", W.rule_sweep("fixed_outdegree", True, scale=0.05), 1 << 21),          # 2e7, 10 blocks
         ("microcircuit", W.microcircuit(scale=0.05), 1 << 16)]                              # 7.5e5, 12 blocks


@pytest.mark.parametrize("name,spec,block", CASES, ids=[c[0] for c in CASES])
def test_block_sorted_build_equals_oracle(snc, oracle_mod, name, spec, block):
    net = snc.Network(spec, block_sort=block).finalize()
    got = net.to_host()
    st = net.stats()
    net.close()
    assert got["src"].size > 4 * block  # several blocks
    assert_network_equal(got, oracle_mod.build(spec), name)
    assert st.source_major == 0


class BudgetAllocator:
    """snc_allocator over torch's caching allocator that refuses any request
    taking the live total above `budget` bytes."""

    def __init__(self, budget, device=0):
        import torch
        from paper_2306_09855_gb300 import snc as mod
        self.torch, self.budget, self.live, self.peak = torch, budget, {}, 0

        def _alloc(nbytes, stream, user):
            if sum(self.live.values()) + nbytes > self.budget:
                return None
            try:
                p = self.torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
            except Exception:
                return None
            self.live[p] = int(nbytes)
            self.peak = max(self.peak, sum(self.live.values()))
            return p

        def _free(ptr, nbytes, stream, user):
            self.live.pop(ptr, None)
            self.torch.cuda.caching_allocator_delete(ptr)

        self._a, self._f = mod.ALLOC_FN(_alloc), mod.FREE_FN(_free)
        self.struct = mod.snc_allocator(self._a, self._f, None)


def test_block_sort_fits_a_budget_the_radix_sort_exceeds(snc, oracle_mod):
    spec = W.two_population(20_000, "fixed_indegree", k=500, autapses=False, seed=3)  # 2e7 connections
    n = 20_000 * 2 * 500 * 2
    budget = int(19 * n)  # bytes: out-of-place sort needs about 26 per connection, the block sort about 14
    default = BudgetAllocator(budget)
    net = snc.Network(spec, allocator=default)
    with pytest.raises(snc.SncError) as e:
        net.finalize()
        net.synchronize()
    assert e.value.name == "OOM"
    net.close()
    blocked = BudgetAllocator(budget)
    net = snc.Network(spec, allocator=blocked, block_sort=1 << 20).finalize()
    got = net.to_host()
    net.close()
    assert blocked.peak <= budget
    assert_network_equal(got, oracle_mod.build(spec), "block sort under a budget")


def test_block_sort_argument_errors(snc):
    import torch
    k = torch.zeros(4096, dtype=torch.int64, device="cuda")
    v = torch.zeros(4096, dtype=torch.int32, device="cuda")
    for block in (0, 1000, 1023):
        with pytest.raises(snc.SncError) as e:
            snc.snc_block_sort_pairs(k.data_ptr(), v.data_ptr(), 4096, 20, block)
        assert e.value.name == "INVALID_ARG"
    big = torch.zeros(257 * 1024, dtype=torch.int64, device="cuda")
    bv = torch.zeros(257 * 1024, dtype=torch.int32, device="cuda")
    with pytest.raises(snc.SncError) as e:
        snc.snc_block_sort_pairs(big.data_ptr(), bv.data_ptr(), 257 * 1024, 20, 1024)
    assert e.value.name == "INVALID_ARG"
    spec = W.plain_indegree()
    net = snc.Network(spec)
    with pytest.raises(snc.SncError) as e:
        snc.snc_set_block_sort(net.ctx, 1500)
    assert e.value.name == "INVALID_ARG"
    snc.snc_set_block_sort(net.ctx, 1024)  # 400,000 connections need 391 blocks of 1024
    with pytest.raises(snc.SncError) as e:
        net.finalize()
    assert e.value.name == "INVALID_ARG"
    net.close()
    a = snc.Network(spec, block_sort=1 << 16)
    b = snc.Network(W.plain_indegree(seed=9))
    with pytest.raises(snc.SncError) as e:
        snc.snc_batch_finalize([a.ctx, b.ctx])
    assert e.value.name == "INVALID_ARG"
    a.close()
    b.close()
    c = snc.Network(spec, block_sort=1 << 16, target_shard=(0, 100))
    with pytest.raises(snc.SncError) as e:
        c.finalize()
    assert e.value.name == "INVALID_ARG"
    c.close()

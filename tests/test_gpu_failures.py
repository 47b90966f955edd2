"""Failure paths of the C ABI on the GPU, reached without faulting it.

- An expired device wait: the test hook snc_set_wait_test withholds one
  tile's look-back words, so that every later tile's bounded wait runs to a
  short limit and sets the device error bit.  The calls report TIMEOUT, and
  the process keeps working: the next build equals the oracle's network.
- A device allocation that fails in the middle of a build: an allocator
  callback that refuses its n-th request.  snc_finalize returns OOM, every
  buffer the build had taken is returned by snc_destroy (none leaks), and a
  fresh context builds the network exactly.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import assert_network_equal
from paper_2306_09855_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09855_gb300 import snc as mod
    mod.load()
    return mod


def _spec():
    return W.two_population(3001, "fixed_indegree", k=97, autapses=False, multapses=True, seed=31)


def test_expired_lookback_wait_reports_timeout_then_builds(snc, oracle_mod):
    spec = _spec()
    try:
        snc.snc_set_wait_test(64, 1)
        net = snc.Network(spec)
        net.finalize()  # queued; the expiry is read back at synchronize
        with pytest.raises(snc.SncError) as e:
            net.synchronize()
        assert e.value.name == "TIMEOUT"
        with pytest.raises(snc.SncError):
            net.view()
        net.close()
    finally:
        snc.snc_set_wait_test()
    net = snc.Network(spec).finalize()
    got = net.to_host()
    net.close()
    assert_network_equal(got, oracle_mod.build(spec), "after timeout")


def test_expired_lookback_wait_in_the_allocating_sort(snc):
    import torch
    rng = np.random.default_rng(5)
    n, bits = 300_000, 27
    keys = rng.integers(0, 1 << bits, n, dtype=np.uint64)
    vals = np.arange(n, dtype=np.uint32)
    kin = torch.from_numpy(keys.view(np.int64)).cuda()
    vin = torch.from_numpy(vals.view(np.int32)).cuda()
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    args = (kin.data_ptr(), vin.data_ptr(), kout.data_ptr(), vout.data_ptr(), n, bits,
            torch.cuda.current_stream().cuda_stream)
    try:
        snc.snc_set_wait_test(32, 0)
        with pytest.raises(snc.SncError) as e:
            snc.snc_radix_sort_pairs(*args)
        assert e.value.name == "TIMEOUT"
    finally:
        snc.snc_set_wait_test()
    snc.snc_radix_sort_pairs(*args)
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(kout.cpu().numpy().view(np.uint64), keys[order])
    np.testing.assert_array_equal(vout.cpu().numpy().view(np.uint32), vals[order])


class FailingAllocator:
    """snc_allocator over torch's caching allocator that refuses request
    number `fail_at` (1-based) and counts the buffers it has handed out."""

    def __init__(self, fail_at, device=0):
        import torch
        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}

        def _alloc(nbytes, stream, user):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            try:
                p = self.torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
            except Exception:
                return None
            self.live[p] = int(nbytes)
            return p

        def _free(ptr, nbytes, stream, user):
            assert ptr in self.live, "free of a buffer this allocator did not hand out"
            assert self.live.pop(ptr) == int(nbytes)
            self.torch.cuda.caching_allocator_delete(ptr)

        from paper_2306_09855_gb300 import snc as mod
        self._a = mod.ALLOC_FN(_alloc)
        self._f = mod.FREE_FN(_free)
        self.struct = mod.snc_allocator(self._a, self._f, None)


def _context(snc, spec, alloc):
    import torch
    cfg = snc.snc_config(seed=spec.seed, dt_ms=spec.dt, device=0, reserved=0,
                         stream=torch.cuda.current_stream().cuda_stream,
                         allocator=ctypes.pointer(alloc.struct))
    ctx = snc.snc_create(cfg)
    for n in spec.populations:
        snc.snc_create_population(ctx, n)
    for pj in spec.projections:
        snc.snc_connect(ctx, snc.snc_range(*pj.src), snc.snc_range(*pj.tgt), snc._rule_struct(pj),
                        snc._syn_struct(pj))
    return ctx


def test_allocation_failure_mid_build_returns_oom_without_leak(snc, oracle_mod):
    spec = W.two_population(2003, "pairwise_bernoulli", p=0.02, autapses=False, multapses=False, seed=8)
    probe = FailingAllocator(fail_at=0)
    ctx = _context(snc, spec, probe)
    snc.snc_finalize(ctx)
    snc.snc_synchronize(ctx)
    total = probe.calls
    snc.snc_destroy(ctx)
    assert total > 5 and not probe.live
    hit = 0
    for k in sorted({1, 2, total // 3, total // 2, total - 1, total}):
        alloc = FailingAllocator(fail_at=k)
        ctx = _context(snc, spec, alloc)
        with pytest.raises(snc.SncError) as e:
            snc.snc_finalize(ctx)
            snc.snc_synchronize(ctx)
        assert e.value.name == "OOM", (k, e.value)
        hit += 1
        snc.snc_destroy(ctx)
        assert not alloc.live, (k, len(alloc.live))
    assert hit >= 3
    net = snc.Network(spec).finalize()
    got = net.to_host()
    net.close()
    assert_network_equal(got, oracle_mod.build(spec), "after OOM")

"""snc_radix_sort_pairs_noalloc against snc_radix_sort_pairs.

The no-allocation variant serves callers that must not allocate device memory
(for example a simulator that has given all of the GPU's memory to its own
pool, or latency-bound code that cannot pay for the device synchronisation an
allocation may cause).  Its working memory is a static device array shared by
all calls, so two calls in a row must still give exactly the result of the
allocating sort (integer keys and values: bit-exact).  Kept in its own file,
collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09855_gb300 import snc
    snc.load()
    return torch, snc


def _sort(torch, fn, keys, vals, bits):
    kin = torch.from_numpy(keys.view(np.int64)).cuda()
    vin = torch.from_numpy(vals.view(np.int32)).cuda()
    kout = torch.empty_like(kin)
    vout = torch.empty_like(vin)
    fn(kin.data_ptr(), vin.data_ptr(), kout.data_ptr(), vout.data_ptr(), keys.size, bits,
       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return kout.cpu().numpy().view(np.uint64), vout.cpu().numpy().view(np.uint32)


def test_noalloc_sort_equals_allocating_sort_on_two_calls(env):
    torch, snc = env
    cases = [(300_001, 43), (snc.SNC_NOALLOC_MAX_PAIRS, 29)]  # four passes, then three
    for call, (n, bits) in enumerate(cases):
        rng = np.random.default_rng(100 + call)
        keys = rng.integers(0, 1 << bits, n, dtype=np.uint64) & ~np.uint64(0xF)  # duplicates
        vals = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
        k_ref, v_ref = _sort(torch, snc.snc_radix_sort_pairs, keys, vals, bits)
        k_got, v_got = _sort(torch, snc.snc_radix_sort_pairs_noalloc, keys, vals, bits)
        np.testing.assert_array_equal(k_got, k_ref)
        np.testing.assert_array_equal(v_got, v_ref)


def test_noalloc_sort_rejects_more_than_its_limit(env):
    torch, snc = env
    n = snc.SNC_NOALLOC_MAX_PAIRS + 1
    k = torch.zeros(n, dtype=torch.int64, device="cuda")
    v = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(snc.SncError) as e:
        snc.snc_radix_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), k.data_ptr(), v.data_ptr(), n, 20)
    assert e.value.name == "INVALID_ARG"
    assert "exceeds" in str(e.value)

"""snc_radix_sort_pairs_noalloc against numpy's stable sort and against
snc_radix_sort_pairs.

The no-allocation variant serves callers that must not allocate device memory
(for example a simulator that has given all of the GPU's memory to its own
pool, or latency-bound code that cannot pay for the device synchronisation an
allocation may cause).  Its working memory is a static device array shared by
all calls, so two calls in a row must still give exactly the stable order of
the keys (integer keys and values: bit-exact).  Kept in its own file,
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


def _stable(keys, vals, bits):
    mask = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    order = np.argsort(keys & mask, kind="stable")
    return keys[order], vals[order]


def _case(seed, n, bits):
    rng = np.random.default_rng(seed)
    hi = 1 << bits if bits < 64 else 1 << 63
    keys = rng.integers(0, hi, n, dtype=np.uint64) & ~np.uint64(0xF)  # duplicates
    if bits == 64:
        keys |= rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)
    vals = np.arange(n, dtype=np.uint32) ^ np.uint32(0x5A5A5A5A)  # distinct: stability shows
    return keys, vals


def test_noalloc_sort_equals_stable_sort_on_two_calls(env):
    torch, snc = env
    # 43-bit keys take five passes of at most 9 bits, then 29-bit keys four.
    cases = [(300_001, 43), (snc.SNC_NOALLOC_MAX_PAIRS, 29)]
    for call, (n, bits) in enumerate(cases):
        keys, vals = _case(100 + call, n, bits)
        k_ref, v_ref = _stable(keys, vals, bits)
        k_got, v_got = _sort(torch, snc.snc_radix_sort_pairs_noalloc, keys, vals, bits)
        np.testing.assert_array_equal(k_got, k_ref)
        np.testing.assert_array_equal(v_got, v_ref)
        k_al, v_al = _sort(torch, snc.snc_radix_sort_pairs, keys, vals, bits)
        np.testing.assert_array_equal(k_al, k_ref)
        np.testing.assert_array_equal(v_al, v_ref)


def test_noalloc_sort_ignores_process_tuning(env):
    """With the widest tuned digit (11 bits) the no-allocation sort keeps its
    own plan and still sorts its largest input, 64-bit keys included."""
    torch, snc = env
    old = snc.snc_get_tuning()
    try:
        snc.snc_set_tuning(sort_digit_bits=11, sort_group_tiles=1, sort_items=16)
        for seed, bits in ((7, 64), (8, 33)):
            keys, vals = _case(seed, snc.SNC_NOALLOC_MAX_PAIRS, bits)
            k_ref, v_ref = _stable(keys, vals, bits)
            k_got, v_got = _sort(torch, snc.snc_radix_sort_pairs_noalloc, keys, vals, bits)
            np.testing.assert_array_equal(k_got, k_ref)
            np.testing.assert_array_equal(v_got, v_ref)
    finally:
        snc.snc_set_tuning(sort_digit_bits=old.sort_digit_bits, sort_group_tiles=old.sort_group_tiles,
                           gen_blocks_per_sm=old.gen_blocks_per_sm, sort_items=old.sort_items)


def test_noalloc_sort_reports_an_expired_wait(env):
    """A look-back wait that runs to its bound (a tile withheld by the test
    hook) is reported as TIMEOUT; the next call sorts correctly."""
    torch, snc = env
    keys, vals = _case(9, 200_000, 30)
    try:
        snc.snc_set_wait_test(64, 1)
        with pytest.raises(snc.SncError) as e:
            _sort(torch, snc.snc_radix_sort_pairs_noalloc, keys, vals, 30)
        assert e.value.name == "TIMEOUT"
    finally:
        snc.snc_set_wait_test()
    k_ref, v_ref = _stable(keys, vals, 30)
    k_got, v_got = _sort(torch, snc.snc_radix_sort_pairs_noalloc, keys, vals, 30)
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

"""The onesweep radix sort on its own (snc_radix_sort_pairs) against numpy's
stable argsort, for several key widths, sizes and tails."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_snc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09855_gb300 import snc
    snc.load()
    return torch, snc


@pytest.mark.parametrize("n,bits", [(1, 5), (100, 8), (6143, 11), (6145, 11), (50_001, 29), (300_000, 43),
                                    (1_000_003, 64), (200_000, 17), (40_000, 1)])
def test_sort_matches_stable_argsort(torch_snc, n, bits):
    torch, snc = torch_snc
    rng = np.random.default_rng(n + bits)
    hi = (1 << bits) if bits < 64 else None
    if hi is None:
        keys = rng.integers(0, 2**63, n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, n, dtype=np.uint64)
    else:
        # many duplicates so that stability matters
        keys = rng.integers(0, min(hi, max(2, n // 3)), n, dtype=np.uint64) * np.uint64(max(1, hi // max(2, n // 3)))
        keys %= np.uint64(hi)
    vals = np.arange(n, dtype=np.uint32)
    kin = torch.from_numpy(keys.view(np.int64)).cuda()
    vin = torch.from_numpy(vals.view(np.int32)).cuda()
    kout = torch.empty_like(kin)
    vout = torch.empty_like(vin)
    snc.snc_radix_sort_pairs(kin.data_ptr(), vin.data_ptr(), kout.data_ptr(), vout.data_ptr(), n, bits,
                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(kout.cpu().numpy().view(np.uint64), keys[order])
    np.testing.assert_array_equal(vout.cpu().numpy().view(np.uint32), vals[order])
    np.testing.assert_array_equal(kin.cpu().numpy().view(np.uint64), keys)  # input untouched


# (digit bits, tiles per look-back unit, keys per thread); the last only
# matters for the bulk-copy kernel (group 0, 8-9 bit digits).
TUNINGS = [(8, 0, 16), (9, 0, 16), (8, 0, 12), (9, 0, 12), (8, 0, 8), (9, 0, 8), (8, 0, 24), (9, 0, 24),
           (8, 0, 32), (9, 0, 32), (8, 1, 16), (9, 4, 16), (9, 8, 16), (10, 8, 16), (11, 4, 16), (11, 8, 16),
           (11, 1, 16)]


def _restore(snc, old):
    snc.snc_set_tuning(sort_digit_bits=old.sort_digit_bits, sort_group_tiles=old.sort_group_tiles,
                       sort_items=old.sort_items)


@pytest.mark.parametrize("bits,group,items", TUNINGS, ids=[f"d{b}g{g}i{i}" for b, g, i in TUNINGS])
def test_every_sort_variant_matches_stable_argsort(torch_snc, bits, group, items):
    """Every kernel variant the tuner can pick gives the stable order."""
    torch, snc = torch_snc
    old = snc.snc_get_tuning()
    try:
        snc.snc_set_tuning(sort_digit_bits=bits, sort_group_tiles=group, sort_items=items)
        for n, kb in ((70_001, 43), (4096 * 9, 20), (1000, 64)):
            rng = np.random.default_rng(n + kb + bits)
            keys = rng.integers(0, 1 << min(kb, 63), n, dtype=np.uint64) & ~np.uint64(0x3F)
            vals = np.arange(n, dtype=np.uint32)
            kin = torch.from_numpy(keys.view(np.int64)).cuda()
            vin = torch.from_numpy(vals.view(np.int32)).cuda()
            kout = torch.empty_like(kin)
            vout = torch.empty_like(vin)
            snc.snc_radix_sort_pairs(kin.data_ptr(), vin.data_ptr(), kout.data_ptr(), vout.data_ptr(), n, kb,
                                     torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            order = np.argsort(keys, kind="stable")
            np.testing.assert_array_equal(kout.cpu().numpy().view(np.uint64), keys[order])
            np.testing.assert_array_equal(vout.cpu().numpy().view(np.uint32), vals[order])
    finally:
        _restore(snc, old)


def test_misaligned_buffers_fall_back(torch_snc):
    """Arrays that are not 16-byte aligned are sorted by the non-bulk-copy path."""
    torch, snc = torch_snc
    old = snc.snc_get_tuning()
    try:
        snc.snc_set_tuning(sort_digit_bits=8, sort_group_tiles=0)
        n = 50_000
        rng = np.random.default_rng(5)
        keys = rng.integers(0, 1 << 30, n + 1, dtype=np.uint64)
        vals = np.arange(n + 1, dtype=np.uint32)
        kin = torch.from_numpy(keys.view(np.int64)).cuda()
        vin = torch.from_numpy(vals.view(np.int32)).cuda()
        kout = torch.empty_like(kin)
        vout = torch.empty_like(vin)
        # offset every pointer by one element: 8 and 4 bytes
        snc.snc_radix_sort_pairs(kin.data_ptr() + 8, vin.data_ptr() + 4, kout.data_ptr() + 8, vout.data_ptr() + 4,
                                 n, 30, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        order = np.argsort(keys[1:], kind="stable")
        np.testing.assert_array_equal(kout.cpu().numpy().view(np.uint64)[1:], keys[1:][order])
        np.testing.assert_array_equal(vout.cpu().numpy().view(np.uint32)[1:], vals[1:][order])
    finally:
        _restore(snc, old)

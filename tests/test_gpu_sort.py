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

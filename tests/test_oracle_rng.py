"""Pins of the oracle's Philox4x32-10 stream against cuRAND's host generator.

cuRAND's CURAND_RNG_PSEUDO_PHILOX4_32_10 host generator (a library routine run
as a black box) is seeded with a 64-bit seed that becomes the Philox key
(seed lo, seed hi).  Its output element A (absolute index, generator offset
included) is word A mod 4 of Philox at counter
(c0, c1) = floor(A / 2^18) as a 64-bit number, c2 = floor(A / 4) mod 2^16, c3 = 0.
That mapping was established by experiment and covers both key words and
the counter words c0, c1 and c2.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest


def _curand():
    names = [ctypes.util.find_library("curand"), "libcurand.so", "libcurand.so.10"]
    for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
              "/usr/local/cuda/targets/x86_64-linux/lib"):
        names.append(os.path.join(d, "libcurand.so"))
    for n in names:
        if not n:
            continue
        try:
            return ctypes.CDLL(n)
        except OSError:
            continue
    return None


def _curand_host_philox(lib, seed, offset, n):
    g = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(g), 161) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(g, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n, np.uint32)
        assert lib.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(g)
    return out


@pytest.mark.parametrize("seed", [0, 1234, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
@pytest.mark.parametrize("offset", [0, 4 * 65536 - 8, 1 << 50, (1 << 50) + 3 * 262144 + 68])
def test_philox_matches_curand_host(oracle_mod, seed, offset):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    n = 4096
    got = _curand_host_philox(lib, seed, offset, n)
    a = np.arange(n, dtype=np.uint64) + np.uint64(offset)
    blk = a // np.uint64(262144)
    sub = (a // np.uint64(4)) % np.uint64(65536)
    ctr = np.stack([blk & np.uint64(0xFFFFFFFF), blk >> np.uint64(32), sub,
                    np.zeros_like(sub)], axis=1).astype(np.uint32)
    ref = oracle_mod.philox(ctr, (seed & 0xFFFFFFFF, seed >> 32))
    word = (a % np.uint64(4)).astype(np.int64)
    np.testing.assert_array_equal(ref[np.arange(n), word], got)


def test_philox_counter_and_key_sensitivity(oracle_mod):
    """Every counter word and key word changes the output (avalanche)."""
    base = np.zeros((1, 4), np.uint32)
    ref = oracle_mod.philox(base, (1, 2))
    for w in range(4):
        c = base.copy()
        c[0, w] = 1
        out = oracle_mod.philox(c, (1, 2))
        diff = np.unpackbits((out ^ ref).view(np.uint8)).sum()
        assert 40 < diff < 88, (w, diff)
    for key in ((0, 2), (1, 3)):
        out = oracle_mod.philox(base, key)
        diff = np.unpackbits((out ^ ref).view(np.uint8)).sum()
        assert 40 < diff < 88

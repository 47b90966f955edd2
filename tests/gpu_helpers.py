"""Shared helpers of the GPU parity tests (comparison only, no method code)."""
import numpy as np

WEIGHT_ULP = 4  # fp32 ulps allowed between the CUDA weights and the oracle's


def ulp_diff(a, b):
    a = np.asarray(a, np.float32).view(np.int32).astype(np.int64)
    b = np.asarray(b, np.float32).view(np.int32).astype(np.int64)
    # map the sign-magnitude order onto a line so that -0 and +0 are adjacent
    a = np.where(a < 0, -(a & 0x7FFFFFFF), a)
    b = np.where(b < 0, -(b & 0x7FFFFFFF), b)
    return np.abs(a - b)


def assert_network_equal(got, ref, what=""):
    n = ref["src"].size
    assert got["src"].size == n, (what, got["src"].size, n)
    for f in ("src", "tgt", "delay"):
        np.testing.assert_array_equal(got[f].astype(np.int64), ref[f].astype(np.int64), err_msg=f"{what}:{f}")
    for f in ("row_ptr", "group_ptr"):
        np.testing.assert_array_equal(got[f].astype(np.int64), ref[f].astype(np.int64), err_msg=f"{what}:{f}")
    assert got["n_groups"] == ref["n_groups"], what
    np.testing.assert_array_equal(got["group_first"][:ref["n_groups"]].astype(np.int64),
                                  ref["group_first"].astype(np.int64), err_msg=f"{what}:group_first")
    if n:
        d = ulp_diff(got["weight"], ref["weight"])
        assert d.max() <= WEIGHT_ULP, (what, int(d.max()))

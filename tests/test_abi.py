"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/*.h declare (no GPU needed: no compute call is made)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    inc = os.path.join(ROOT, "include")
    text = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    return sorted(set(re.findall(r"^\s*(?:snc_status|const char\*)\s+(snc_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("snc_create", "snc_destroy", "snc_create_population", "snc_connect",
                 "snc_finalize", "snc_synchronize", "snc_get_connections",
                 "snc_copy_connections", "snc_last_error", "snc_radix_sort_pairs"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2306_09855_gb300 import snc
    lib = snc.load()
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(snc.EXPORTS) == _declared()


def test_last_error_without_context():
    from paper_2306_09855_gb300 import snc
    assert isinstance(snc.snc_last_error(None), str)


def test_sort_argument_checks_need_no_gpu():
    from paper_2306_09855_gb300 import snc
    with pytest.raises(snc.SncError) as e:
        snc.snc_radix_sort_pairs(0, 0, 0, 0, 10, 0)
    assert e.value.name == "INVALID_ARG"
    snc.snc_radix_sort_pairs(0, 0, 0, 0, 0, 12)  # empty input: nothing to do


def test_server_config_checks_need_no_gpu():
    from paper_2306_09855_gb300 import snc
    for kw in ({"hbm_budget_bytes": 0}, {"hbm_budget_bytes": 1 << 30, "max_slots": 0},
               {"hbm_budget_bytes": 1 << 30, "max_slots": 65},
               {"hbm_budget_bytes": 1 << 30, "batch_max_nets": 0},
               {"hbm_budget_bytes": 1 << 30, "batch_max_nets": 257}):
        with pytest.raises(snc.SncError) as e:
            snc.snc_server_create(**kw)
        assert e.value.name == "INVALID_ARG"
    for call in (lambda: snc.snc_server_submit(None, None), lambda: snc.snc_server_wait_any(None),
                 lambda: snc.snc_server_get_stats(None), lambda: snc.snc_server_release(None, 1)):
        with pytest.raises(snc.SncError) as e:
            call()
        assert e.value.name == "INVALID_ARG"
    snc.snc_server_destroy(None)


def test_tuning_ranges_need_no_gpu():
    from paper_2306_09855_gb300 import snc
    old = snc.snc_get_tuning()
    try:
        for items in (8, 12, 16, 24, 32):
            snc.snc_set_tuning(sort_items=items)
            assert snc.snc_get_tuning().sort_items == items
        for bad in ({"sort_items": 20}, {"sort_items": 64}, {"sort_digit_bits": 12}, {"sort_group_tiles": 3},
                    {"gen_blocks_per_sm": 0}):
            with pytest.raises(snc.SncError) as e:
                snc.snc_set_tuning(**bad)
            assert e.value.name == "INVALID_ARG"
    finally:
        snc.snc_set_tuning(sort_digit_bits=old.sort_digit_bits, sort_group_tiles=old.sort_group_tiles,
                           gen_blocks_per_sm=old.gen_blocks_per_sm, sort_items=old.sort_items)


def test_deliver_argument_checks_need_no_gpu():
    from paper_2306_09855_gb300 import snc
    with pytest.raises(snc.SncError) as e:
        snc.snc_deliver(None, 0, 0, 0, 10, 0)
    assert e.value.name == "INVALID_ARG"

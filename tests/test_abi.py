"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/snc.h declares (no GPU needed: no compute call is made)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "snc.h")).read()
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

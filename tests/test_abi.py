"""The C ABI library loads and exports every entry point declared in
include/*.h (no GPU needed; no compute call is made)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_17461_gb300 import build

    build.build()
    from paper_2306_17461_gb300 import binding

    return binding.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for mt in re.finditer(r"\b(?:int|uint64_t|const char \*|void)\s*\*?\s*(ed_\w+)\s*\(", src):
            names.add(mt.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for need in ["ed_create", "ed_distance", "ed_submit", "ed_poll", "ed_destroy", "ed_strerror",
                 "ed_distance_dev", "ed_distance_batch_dev", "ed_prefix_hash_dev", "ed_lcp_dev"]:
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_strerror_and_defaults(lib):
    from paper_2306_17461_gb300 import binding as ed

    assert ed.ed_strerror(0) == "ok"
    assert "invalid" in ed.ed_strerror(ed.ED_EINVAL)
    assert ed.ed_strerror(12345) == "unknown status"
    c = ed.ed_config_default()
    assert c.device == -1 and c.spin_limit_ns == 2_000_000_000 and c.lcp_mode == ed.ED_LCP_AUTO


def test_invalid_arguments_rejected_before_any_cuda_call(lib):
    k = ctypes.c_uint64()
    assert lib.ed_distance(None, None, 0, None, 0, ctypes.byref(k)) == -1
    assert lib.ed_create(None, None) == -1
    assert lib.ed_poll(None, 1, ctypes.byref(k)) == -1
    assert lib.ed_destroy(None) == -1

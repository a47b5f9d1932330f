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


def test_binding_structs_match_the_header(tmp_path):
    """Field offsets and sizes of ed_config and ed_stats as a C compiler lays
    them out from include/ed.h equal the ctypes structures of the binding."""
    import shutil
    import subprocess

    from paper_2306_17461_gb300 import binding as ed

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ed.h"', "int main(void) {"]
    for sname, cls in [("ed_config", ed.ed_config), ("ed_stats", ed.ed_stats)]:
        lines.append(f'printf("{sname} size %zu\\n", sizeof({sname}));')
        for f in cls._fields_:
            lines.append(f'printf("{sname} {f[0]} %zu\\n", offsetof({sname}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for sname, cls in [("ed_config", ed.ed_config), ("ed_stats", ed.ed_stats)]:
        assert got[(sname, "size")] == ctypes.sizeof(cls), sname
        for f in cls._fields_:
            assert got[(sname, f[0])] == getattr(cls, f[0]).offset, (sname, f[0])

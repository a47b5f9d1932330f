"""The tuning table's lookup (host only, no GPU): rows are chosen by the
longer string's length and the expected edit rate, the first matching row
wins, a missing hint counts as an edit rate of 1e-4, and unreadable or
malformed tables and lengths no row covers are refused.  The committed
table (written by the sweep in paper_2306_17461_gb300/tune.py from GB300
measurements) parses and covers the lengths it was measured on."""
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLE = os.path.join(ROOT, "paper_2306_17461_gb300", "tune_table.tsv")


@pytest.fixture()
def ed():
    from paper_2306_17461_gb300 import binding
    from paper_2306_17461_gb300 import build

    build.build()
    binding.load()
    return binding


def _write(tmp_path, text):
    p = tmp_path / "t.tsv"
    p.write_text(text)
    return str(p)


def test_rows_by_length_and_rate(ed, tmp_path):
    t = _write(tmp_path, """# n_lo n_hi rate_lo rate_hi lcp h s0 warp_cap local help
0     1e7  0     1e-3  1 16 64 4096 1 8   # short, few edits
0     1e7  1e-3  1     1 8  32 2048 0 0   # short, many edits
1e7   1e12 0     1     2 4  256 16384 4 4 # long: hash
""")
    c = ed.ed_tune_lookup(10**6, 10**6, 100, t)
    assert (c.lcp_mode, c.block_rounds, c.tile_width, c.warp_cap, c.local_chunks, c.help_div) == (1, 16, 64, 4096, 1, 8)
    c = ed.ed_tune_lookup(10**6, 900_000, 10**4, t)  # rate 1e-2
    assert (c.block_rounds, c.tile_width, c.warp_cap, c.local_chunks, c.help_div) == (8, 32, 2048, -1, -1)
    c = ed.ed_tune_lookup(5, 2 * 10**7, 0, t)  # the longer string decides
    assert (c.lcp_mode, c.block_rounds, c.tile_width) == (2, 4, 256)
    c = ed.ed_tune_lookup(10**6, 10**6, 0, t)  # no hint: rate 1e-4
    assert c.block_rounds == 16
    # the fields the row does not set keep their defaults
    assert c.hash_block == 0 and c.max_inflight == 1024


def test_first_matching_row_wins(ed, tmp_path):
    t = _write(tmp_path, "0 1e9 0 1 1 8 64 4096 1 8\n0 1e9 0 1 3 4 64 4096 1 8\n")
    assert ed.ed_tune_lookup(1000, 1000, 5, t).block_rounds == 8


def test_refusals(ed, tmp_path):
    with pytest.raises(ed.EdError) as e:
        ed.ed_tune_lookup(10, 10, 0, str(tmp_path / "missing.tsv"))
    assert e.value.code == ed.ED_EINVAL
    bad = _write(tmp_path, "0 1e9 0 1 1 8 64\n")  # too few columns
    with pytest.raises(ed.EdError) as e:
        ed.ed_tune_lookup(10, 10, 0, bad)
    assert e.value.code == ed.ED_EINVAL
    out_of_range = _write(tmp_path, "0 1e9 0 1 1 99 64 4096 1 8\n")  # block_rounds > 64
    with pytest.raises(ed.EdError) as e:
        ed.ed_tune_lookup(10, 10, 0, out_of_range)
    assert e.value.code == ed.ED_EINVAL
    narrow = _write(tmp_path, "0 100 0 1 1 8 64 4096 1 8\n")
    with pytest.raises(ed.EdError) as e:
        ed.ed_tune_lookup(1000, 1000, 0, narrow)
    assert e.value.code == ed.ED_ENOTFOUND


@pytest.mark.skipif(not os.path.exists(TABLE), reason="no committed table")
def test_committed_table(ed):
    for n, k in [(10**6, 100), (10**8, 10), (10**8, 10**3), (10**8, 10**5), (10**9, 10**4)]:
        c = ed.ed_tune_lookup(n, n, k, TABLE)
        assert c.lcp_mode in (1, 2, 3) and 1 <= c.block_rounds <= 64
    # the default path of the library is the same file
    assert ed.ed_tune_lookup(10**8, 10**8, 10**3).block_rounds == ed.ed_tune_lookup(10**8, 10**8, 10**3,
                                                                                    TABLE).block_rounds

"""The tuner (host logic, no GPU): the coordinate descent (the value kept per
parameter, the repeated passes, one measurement per setting), and the table
it writes (a row per length and rate bucket, filled by the nearest measured
rate), read back through the library's lookup."""
from collections import Counter

import pytest

from paper_2306_17461_gb300.tune import descend

CANDS = {"h": [8, 16, 32], "d": [8, 2]}


def _cost(table, calls):
    def cost(s):
        key = (s["h"], s["d"])
        calls[key] += 1
        return table[key], key
    return cost


def test_separable_cost_needs_one_pass():
    table = {(h, d): abs(h - 16) + d for h in CANDS["h"] for d in CANDS["d"]}
    calls = Counter()
    best, t, measured = descend(_cost(table, calls), {"h": 32, "d": 8}, CANDS, passes=3)
    assert best == {"h": 16, "d": 2} and t == 2
    assert measured[0][0] == {"h": 32, "d": 8}  # the start first
    assert max(calls.values()) == 1  # every setting once
    # pass one: h 8, h 16, then d 2 from h 16; pass two finds nothing new
    assert [m[2] for m in measured] == [(32, 8), (8, 8), (16, 8), (16, 2), (8, 2), (32, 2)]


def test_interaction_needs_a_second_pass():
    # 16 and 32 rounds a block nearly tie with d = 8; 32 wins only with d = 2
    table = {(8, 8): 15.6, (16, 8): 14.45, (32, 8): 14.52,
             (8, 2): 15.0, (16, 2): 13.51, (32, 2): 12.82}
    one, t1, _ = descend(_cost(table, Counter()), {"h": 32, "d": 8}, CANDS, passes=1)
    assert one == {"h": 16, "d": 2} and t1 == 13.51
    calls = Counter()
    two, t2, measured = descend(_cost(table, calls), {"h": 32, "d": 8}, CANDS, passes=3)
    assert two == {"h": 32, "d": 2} and t2 == 12.82
    assert max(calls.values()) == 1 and len(measured) == len(table)


def test_skip_leaves_values_out():
    table = {(h, d): float(h + d) for h in CANDS["h"] for d in CANDS["d"]}
    calls = Counter()
    best, _, _ = descend(_cost(table, calls), {"h": 32, "d": 8}, CANDS, passes=2,
                         skip=lambda key, v: key == "h")
    assert best == {"h": 32, "d": 2}
    assert set(calls) == {(32, 8), (32, 2)}


P1 = {"lcp_mode": 1, "block_rounds": 16, "tile_width": 64, "warp_cap": 2048, "local_chunks": -1, "help_div": 8}
P2 = {"lcp_mode": 1, "block_rounds": 64, "tile_width": 16, "warp_cap": 16384, "local_chunks": 2, "help_div": -1}
P3 = {"lcp_mode": 1, "block_rounds": 32, "tile_width": 64, "warp_cap": 2048, "local_chunks": -1, "help_div": 2}


def test_table_rows_fill_each_length_bucket_by_nearest_rate():
    from paper_2306_17461_gb300.tune import R_EDGES, table_rows

    best = {(10**6, 1e-6): (P1, 1.0, 1.0), (10**6, 1e-3): (P2, 1.0, 1.0), (10**9, 1e-5): (P3, 1.0, 1.0)}
    rows = table_rows(best)
    # two measured length buckets (no row for the lengths in between), every rate bucket
    assert [(r[0], r[1]) for r in rows] == [(0, 3e6)] * 4 + [(3e8, 1e12)] * 4
    assert [(r[2], r[3]) for r in rows[:4]] == list(zip(R_EDGES[:-1], R_EDGES[1:]))
    # rates up to about 3e-5 take the 1e-6 class, above it the 1e-3 class
    assert [r[4] for r in rows[:4]] == [P1, P1, P2, P2]
    assert all(r[4] == P3 for r in rows[4:])


def test_written_table_is_what_the_library_reads(tmp_path, monkeypatch):
    from paper_2306_17461_gb300 import binding, build, tune

    build.build()
    binding.load()
    monkeypatch.setattr(tune, "HERE", str(tmp_path))
    best = {(10**6, 1e-6): (P1, 1.0, 1.0), (10**6, 1e-3): (P2, 1.0, 1.0), (10**9, 1e-5): (P3, 1.0, 1.0)}
    tune.write([("w", 10**6, 1, P1, 1.0)], best, "test")
    table = str(tmp_path / "tune_table.tsv")
    for n, k, p in [(10**6, 1, P1), (2 * 10**6, 2000, P2), (10**9, 10**4, P3), (5 * 10**8, 10**6, P3)]:
        c = binding.ed_tune_lookup(n, n, k, table)
        got = (c.lcp_mode, c.block_rounds, c.tile_width, c.warp_cap, c.local_chunks, c.help_div)
        # the table keeps "none" (-1) as 0 for local_chunks and help_div; the
        # lookup hands 0 back as -1 (the configuration's explicit none)
        want = tuple(p[x] for x in ("lcp_mode", "block_rounds", "tile_width", "warp_cap")) + \
            tuple(-1 if p[x] <= 0 else p[x] for x in ("local_chunks", "help_div"))
        assert got == want, (n, k, got, want)
    with pytest.raises(binding.EdError):  # lengths between the measured buckets: no row
        binding.ed_tune_lookup(10**7, 10**7, 100, table)

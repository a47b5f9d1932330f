"""The tuner's coordinate descent (host logic, no GPU): the value kept per
parameter, the repeated passes, one measurement per setting."""
from collections import Counter

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

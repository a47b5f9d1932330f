"""Pins for the CPU oracle (no GPU).

The paper prints no numeric worked example, so the oracle is pinned to
things fixed by the mathematics rather than to itself:

* textbook worked examples (tests/golden/levenshtein_textbook.tsv);
* a brute-force breadth-first search over edit scripts (the definition of
  the distance as the fewest single-character edits, Sec. 2), independent
  of any recurrence;
* Algorithm 1 against the DP on every pair of strings up to length 8 over
  {a, b} and on random pairs;
* the frontier definition f_t[i] = max{x : G[x][x-i] <= t} read off the
  full DP table (Appendix A);
* metric invariants and planted-edit bounds.
"""
import itertools
import os
from collections import deque

import numpy as np
import pytest

from paper_2306_17461_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "levenshtein_textbook.tsv")


def _golden():
    rows = []
    with open(GOLDEN, encoding="utf-8") as f:
        for line in f:
            if line.startswith("#") or not line.strip("\n"):
                continue
            a, b, k = line.rstrip("\n").split("\t")
            rows.append((a, b, int(k)))
    return rows


@pytest.mark.parametrize("a,b,k", _golden())
def test_textbook_examples(orc, a, b, k):
    assert orc.dp(a, b) == k
    assert orc.lv(a, b) == k


def _bfs_distances(source: str, alphabet: str, max_len: int) -> dict:
    """Fewest single-character edits from ``source`` to every string of
    length <= max_len, by breadth-first search over the edit graph."""
    dist = {source: 0}
    q = deque([source])
    while q:
        s = q.popleft()
        d = dist[s]
        nbrs = []
        for p in range(len(s)):
            nbrs.append(s[:p] + s[p + 1:])  # deletion
            for c in alphabet:
                if c != s[p]:
                    nbrs.append(s[:p] + c + s[p + 1:])  # substitution
        if len(s) < max_len:
            for p in range(len(s) + 1):
                for c in alphabet:
                    nbrs.append(s[:p] + c + s[p:])  # insertion
        for t in nbrs:
            if t not in dist:
                dist[t] = d + 1
                q.append(t)
    return dist


def test_dp_equals_edit_script_bfs_exhaustive(orc):
    """Every pair of strings of length <= 4 over {a,b,c}; the BFS may pass
    through strings one longer than either end."""
    alphabet = "abc"
    strings = [""] + ["".join(p) for L in range(1, 5) for p in itertools.product(alphabet, repeat=L)]
    pairs, expect = [], []
    for s in strings:
        dist = _bfs_distances(s, alphabet, 5)
        for t in strings:
            pairs.append((s, t))
            expect.append(dist[t])
    got_dp = orc.many("dp", pairs)
    got_lv = orc.many("lv", pairs)
    assert np.array_equal(got_dp, np.array(expect))
    assert np.array_equal(got_lv, np.array(expect))


def test_dp_equals_edit_script_bfs_length5_sample(orc):
    alphabet = "abc"
    rng = np.random.default_rng(5)
    strings = ["".join(p) for p in itertools.product(alphabet, repeat=5)]
    for s in [strings[i] for i in rng.choice(len(strings), 6, replace=False)]:
        dist = _bfs_distances(s, alphabet, 6)
        targets = [strings[i] for i in rng.choice(len(strings), 40, replace=False)]
        for t in targets:
            assert orc.dp(s, t) == dist[t]


def test_lv_equals_dp_every_pair_up_to_8_over_ab(orc):
    strings = [""] + ["".join(p) for L in range(1, 9) for p in itertools.product("ab", repeat=L)]
    assert len(strings) == 511
    pairs = [(s, t) for s in strings for t in strings]
    dp = orc.many("dp", pairs)
    lv = orc.many("lv", pairs)
    assert np.array_equal(dp, lv)
    # spot values fixed by hand
    idx = {s: i for i, s in enumerate(strings)}
    assert dp[idx["ab"] * 511 + idx["ba"]] == 2
    assert dp[idx["aaaa"] * 511 + idx[""]] == 4
    assert dp[idx["abab"] * 511 + idx["baba"]] == 2


@pytest.mark.parametrize("sigma", [2, 4, 256])
def test_lv_equals_dp_random(orc, sigma):
    rng = np.random.default_rng(100 + sigma)
    pairs = []
    for _ in range(60):
        n = int(rng.integers(0, 2000))
        k = int(rng.integers(0, max(1, n // 4) + 1))
        A, B = W.random_pair(rng, n, k, sigma)
        pairs.append((A, B))
    # also fully random (unrelated) pairs of different lengths
    for _ in range(20):
        pairs.append((rng.integers(0, sigma, int(rng.integers(0, 300)), dtype=np.uint8),
                      rng.integers(0, sigma, int(rng.integers(0, 300)), dtype=np.uint8)))
    assert np.array_equal(orc.many("dp", pairs), orc.many("lv", pairs))


def _canonical_frontier(G: np.ndarray, t: int, i: int) -> int | None:
    """max{x : G[x][x-i] <= t} over cells of the grid, None if no cell."""
    n, m = G.shape[0] - 1, G.shape[1] - 1
    best = None
    for x in range(max(0, i), min(n, m + i) + 1):
        if G[x, x - i] <= t:
            best = x
    return best


def test_frontier_matches_definition(orc):
    rng = np.random.default_rng(7)
    for trial in range(40):
        n = int(rng.integers(0, 40))
        sigma = [2, 3, 4][trial % 3]
        A, B = W.random_pair(rng, n, int(rng.integers(0, 8)), sigma)
        G = orc.dp_table(A, B)
        k = int(G[-1, -1])
        kk, F = orc.lv_frontiers(A, B, k)
        assert kk == k
        for t in range(k + 1):
            for i in range(-t, t + 1):
                want = _canonical_frontier(G, t, i)
                got = F[t, i + k]
                if want is None:
                    assert got == orc.NEG, (trial, t, i)
                else:
                    assert got == want, (trial, t, i, got, want)


def test_invariants(orc):
    rng = np.random.default_rng(11)
    for _ in range(30):
        sigma = int(rng.choice([2, 4, 26]))
        A, B = W.random_pair(rng, int(rng.integers(0, 400)), int(rng.integers(0, 30)), sigma)
        C, _ = W.random_pair(rng, int(rng.integers(0, 400)), 0, sigma)
        dab, dba = orc.dp(A, B), orc.dp(B, A)
        assert orc.dp(A, A) == 0
        assert dab == dba
        assert abs(A.size - B.size) <= dab <= max(A.size, B.size)
        assert orc.dp(A, C) <= dab + orc.dp(B, C)
        if A.size == B.size:
            assert dab <= int(np.count_nonzero(A != B))


def test_planted_edit_bounds(orc):
    for idx in range(20):
        p = W.make_pair(90, 3000, 1 + idx * 3, sigma=4, extra=idx)
        k = orc.lv(p.A, p.B)
        assert abs(p.A.size - p.B.size) <= k <= p.edits
        assert k == orc.dp(p.A, p.B)


def test_single_edit_is_distance_one(orc):
    rng = np.random.default_rng(3)
    sym = W.Symbols(4)
    for _ in range(50):
        A = sym.draw(rng, int(rng.integers(1, 200)))
        B = W.plant(rng, A, np.array([int(rng.integers(0, A.size))]), sym)
        assert orc.lv(A, B) == 1 == orc.dp(A, B)


def test_lv_parallel_matches_sequential(orc):
    p = W.make_pair(91, 200000, 3000, sigma=4)
    k1, r1, e1 = orc.lv(p.A, p.B, with_stats=True)
    k2, r2, e2 = orc.lv(p.A, p.B, nthreads=4, with_stats=True)
    assert k1 == k2 == r1 == r2
    assert e1 == e2
    # extensions: sum over rounds of the valid diagonals in [-t, t]
    n, m = p.A.size, p.B.size
    assert e1 == sum(min(t, m) + min(t, n) + 1 for t in range(k1 + 1))


def test_max_rounds_stops_early(orc):
    p = W.make_pair(92, 5000, 200, sigma=4)
    k = orc.lv(p.A, p.B)
    r, rounds, ext = orc.lv(p.A, p.B, max_rounds=k // 2, with_stats=True)
    assert r == -1 and rounds == k // 2


def test_empty_and_degenerate(orc):
    assert orc.lv(b"", b"") == 0
    assert orc.lv(b"", b"xyz") == 3
    assert orc.lv(b"xyzw", b"") == 4
    assert orc.lv(b"aaaa", b"aaaa") == 0
    assert orc.lv(b"aaaa", b"bbbb") == 4
    assert orc.lv(bytes(range(256)), bytes(range(255, -1, -1))) == orc.dp(bytes(range(256)), bytes(range(255, -1, -1)))
    # NUL bytes are ordinary symbols
    assert orc.lv(b"\x00\x00\x01", b"\x00\x01") == 1


def test_lcp_definition(orc):
    a = np.frombuffer(b"abcabcabd", dtype=np.uint8)
    b = np.frombuffer(b"abcabd", dtype=np.uint8)
    assert orc.lcp(a, b, 0, 0) == 5
    assert orc.lcp(a, b, 3, 0) == 6  # "abcabd" vs "abcabd"
    assert orc.lcp(a, b, 3, 3) == 2
    assert orc.lcp(a, b, 9, 0) == 0
    assert orc.lcp(a, b, 0, 6) == 0

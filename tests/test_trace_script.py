"""The edit-script traceback (host code of the C ABI) on the oracle's own
frontiers, no GPU: for random, planted and degenerate pairs the script it
returns turns A into B with matching characters between operations and
has exactly the oracle's distance of operations, hence is optimal; and
frontiers that describe no such alignment are refused."""
import numpy as np
import pytest

from gpu_util import mirror_oracle_frontier
from paper_2306_17461_gb300 import workloads as W
from script_check import script_transforms


def _trace(orc, A, B, slack=2):
    from paper_2306_17461_gb300 import binding as ed

    k = orc.lv(A, B)
    T = k + slack
    ko, Fo = orc.lv_frontiers(A, B, T)
    assert ko == k
    F = mirror_oracle_frontier(Fo, T, orc.NEG, ed.NEG32).astype(np.int32)
    return k, ed.ed_trace_script(F, T, len(A), len(B), k)


def test_random_pairs(orc):
    rng = np.random.default_rng(41)
    for trial in range(60):
        sigma = [2, 4, 256][trial % 3]
        A, B = W.random_pair(rng, int(rng.integers(0, 400)), int(rng.integers(0, 40)), sigma)
        k, ops = _trace(orc, A, B)
        assert len(ops) == k
        assert script_transforms(A, B, ops), trial


def test_every_short_binary_pair(orc):
    # all pairs of binary strings of length <= 4 (341 x 341 would be slow in
    # Python; lengths 0..4 on both sides give 31 x 31 pairs)
    strs = [np.array([(v >> i) & 1 for i in range(L)], dtype=np.uint8) for L in range(5) for v in range(2**L)]
    for A in strs:
        for B in strs:
            k, ops = _trace(orc, A, B)
            assert len(ops) == k and script_transforms(A, B, ops)


def test_degenerate_pairs(orc):
    x = np.random.default_rng(42).integers(0, 4, 200, dtype=np.uint8)
    empty = np.zeros(0, np.uint8)
    for A, B in [(x, x), (x, empty), (empty, x), (empty, empty), (x, x + 4),
                 (np.zeros(50, np.uint8), np.zeros(20, np.uint8))]:
        k, ops = _trace(orc, A, B)
        assert len(ops) == k and script_transforms(A, B, ops)


def test_inconsistent_frontiers_are_refused(orc):
    from paper_2306_17461_gb300 import binding as ed

    A = np.frombuffer(b"kitten", dtype=np.uint8)
    B = np.frombuffer(b"sitting", dtype=np.uint8)
    k = orc.lv(A, B)
    ko, Fo = orc.lv_frontiers(A, B, k)
    F = mirror_oracle_frontier(Fo, k, orc.NEG, ed.NEG32).astype(np.int32)
    # a claimed distance below the true one: no alignment reaches (n, m)
    with pytest.raises(ed.EdError) as e:
        ed.ed_trace_script(F, k, len(A), len(B), k - 1)
    assert e.value.code == ed.ED_EINVAL
    # a frontier row wiped out
    G = F.copy()
    G[k - 1, :] = ed.NEG32
    with pytest.raises(ed.EdError):
        ed.ed_trace_script(G, k, len(A), len(B), k)

"""Pins for the oracle's prefix hash and hash LCP (Sec. 2, Sec. 3.2).

The prefix table is checked against Python's arbitrary-precision integers
evaluating the defining sum directly (not Horner's rule), and against the
concatenation identity h([S1,S2]) = h(S1) * p^|S2| + h(S2) of Sec. 2.  The
hash LCP is checked against the character-by-character LCP.
"""
import numpy as np
import pytest

Q = (1 << 61) - 1


def _sum_hash(x: bytes, base: int) -> int:
    L = len(x)
    return sum((c + 1) * pow(base, L - 1 - j, Q) for j, c in enumerate(x)) % Q


@pytest.mark.parametrize("base", [257, 1000003, Q - 2, (1 << 40) + 15])
def test_prefix_hash_definition(orc, base):
    rng = np.random.default_rng(base % 1000)
    X = rng.integers(0, 256, 300, dtype=np.uint8)
    T = orc.prefix_hash(X, base)
    assert T[0] == 0
    xb = X.tobytes()
    for x in [0, 1, 2, 3, 17, 64, 255, 299, 300]:
        assert int(T[x]) == _sum_hash(xb[:x], base), x


def test_prefix_hash_long_horner_vs_bigint(orc):
    rng = np.random.default_rng(1)
    X = rng.integers(0, 4, 100000, dtype=np.uint8)
    base = 1234567891011
    T = orc.prefix_hash(X, base)
    h = 0
    for j, c in enumerate(X.tolist()):
        h = h * base + c + 1  # exact integer, reduced only at checkpoints
        if (j + 1) % 9973 == 0 or j + 1 == X.size:
            assert int(T[j + 1]) == h % Q
            h %= Q


def test_concatenation_identity(orc):
    rng = np.random.default_rng(2)
    base = 987654321987
    for _ in range(50):
        L = int(rng.integers(2, 500))
        X = rng.integers(0, 256, L, dtype=np.uint8)
        T = orc.prefix_hash(X, base)
        s = int(rng.integers(1, L))
        h1 = int(T[s])
        h2 = orc.range_hash(T, s, L - s, base)
        assert (h1 * pow(base, L - s, Q) + h2) % Q == int(T[L])
        assert h2 == _sum_hash(X[s:].tobytes(), base)


def test_mulmod_edge_values(orc):
    # T[1] = (0 * base + c + 1) and T[2] = (T[1] * base + c + 1) mod Q at the
    # largest bases exercise the 128-bit product and the reduction.
    for base in [Q - 1, Q - 2, 2**60, 2**61 - 3]:
        X = np.array([255, 255, 0, 128], dtype=np.uint8)
        T = orc.prefix_hash(X, base)
        h = 0
        for j, c in enumerate(X.tolist()):
            h = (h * base + c + 1) % Q
            assert int(T[j + 1]) == h
    assert orc.powmod(3, 0) == 1
    assert orc.powmod(Q - 1, 2) == 1  # (-1)^2
    assert orc.powmod(2, 61) == 1     # 2^61 = 1 mod 2^61-1


def test_hash_lcp_equals_direct_lcp(orc):
    rng = np.random.default_rng(4)
    base = (1 << 45) + 59
    for sigma in [2, 4, 256]:
        A = rng.integers(0, sigma, 3000, dtype=np.uint8)
        B = A.copy()
        # plant a few mismatches so there are long and short common runs
        for p in rng.choice(3000, 12, replace=False):
            B[p] = (int(B[p]) + 1) % sigma
        TA, TB = orc.prefix_hash(A, base), orc.prefix_hash(B, base)
        for _ in range(300):
            x = int(rng.integers(0, 3001))
            y = x if rng.random() < 0.6 else int(rng.integers(0, 3001))
            assert orc.hash_lcp(TA, A.size, TB, B.size, base, x, y) == orc.lcp(A, B, x, y)

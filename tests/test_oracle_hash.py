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


# ---------------------------------------------------------------- blocked
# Sec. 3.3 / Alg. 2: the table keeps the prefixes of whole blocks only, and
# GetHash extends the last one by the characters after it.

@pytest.mark.parametrize("b", [1, 2, 7, 32, 64, 500])
def test_blocked_table_definition(orc, b):
    """TB[j] is the defining sum over X[0..j*b), in Python integers (the
    oracle builds it differently: block hashes joined by a scan)."""
    base = 1000003
    rng = np.random.default_rng(b)
    X = rng.integers(0, 256, 333, dtype=np.uint8)
    TB = orc.prefix_hash_blocked(X, b, base)
    assert TB.size == X.size // b + 1 and TB[0] == 0
    xb = X.tobytes()
    for j in range(TB.size):
        assert int(TB[j]) == _sum_hash(xb[:j * b], base), (b, j)


@pytest.mark.parametrize("b", [1, 3, 32])
def test_blocked_table_is_the_full_table_every_b(orc, b):
    base = 257
    rng = np.random.default_rng(5 + b)
    X = rng.integers(0, 4, 5000, dtype=np.uint8)
    T = orc.prefix_hash(X, base)
    TB = orc.prefix_hash_blocked(X, b, base)
    assert np.array_equal(TB, T[::b][:TB.size])


@pytest.mark.parametrize("b", [1, 5, 32])
def test_get_hash_blocked_every_prefix(orc, b):
    """GetHash(i) = h(X[0..i)) for every i, block boundaries and the string
    end included (against the defining sum on a short string, against the
    full table on a longer one)."""
    base = (1 << 40) + 15
    rng = np.random.default_rng(11 * b)
    X = rng.integers(0, 256, 97, dtype=np.uint8)
    TB = orc.prefix_hash_blocked(X, b, base)
    xb = X.tobytes()
    for i in range(X.size + 1):
        assert orc.get_hash_blocked(X, TB, b, base, i) == _sum_hash(xb[:i], base), (b, i)
    Y = rng.integers(0, 3, 4000, dtype=np.uint8)
    T = orc.prefix_hash(Y, base)
    TBy = orc.prefix_hash_blocked(Y, b, base)
    for i in rng.integers(0, Y.size + 1, 300):
        assert orc.get_hash_blocked(Y, TBy, b, base, int(i)) == int(T[int(i)])


def test_blocked_string_shorter_than_a_block(orc):
    X = np.arange(10, dtype=np.uint8)
    TB = orc.prefix_hash_blocked(X, 32, 257)
    assert TB.tolist() == [0]
    assert orc.get_hash_blocked(X, TB, 32, 257, 0) == 0
    assert orc.get_hash_blocked(X, TB, 32, 257, 10) == _sum_hash(X.tobytes(), 257)


@pytest.mark.parametrize("b", [1, 32])
def test_blocked_hash_lcp_equals_direct_lcp(orc, b):
    """The search on blocked tables finds the character LCP (no collision
    on these inputs), including LCPs that cross many blocks and end at a
    string end."""
    base = 1000003
    rng = np.random.default_rng(40 + b)
    n = 3000
    A = rng.integers(0, 2, n, dtype=np.uint8)
    B = A.copy()
    flips = rng.choice(n, 40, replace=False)
    B[flips] ^= 1
    TA = orc.prefix_hash_blocked(A, b, base)
    TB = orc.prefix_hash_blocked(B, b, base)
    for _ in range(300):
        x = int(rng.integers(0, n + 1))
        y = min(n, max(0, x + int(rng.integers(-3, 4))))
        want = orc.lcp(A, B, x, y)
        assert orc.hash_lcp_blocked(A, TA, B, TB, b, base, x, y) == want, (x, y)

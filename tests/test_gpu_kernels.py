"""Building blocks on the GPU against the oracle: the LCP slides (per
thread, per warp with ballot/first-set-bit, whole grid), the prefix-hash
scan and the hash LCP (Sec. 2, Sec. 3.2).  All integer work: bit-exact."""
import numpy as np
import pytest

from gpu_util import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2306_17461_gb300 import binding as ed

    assert torch.cuda.is_available()
    c = ed.Context(device=0)
    yield c
    c.close()


def _lcp_cases(rng):
    """Strings with planted mismatches and queries at every alignment pair
    (x mod 16, y mod 16), near both ends and past them."""
    n = 5000
    A = rng.integers(0, 4, n, dtype=np.uint8)
    B = A.copy()
    for p in rng.choice(n, 25, replace=False):
        B[p] = (B[p] + 1) % 4
    xs, ys = [], []
    for base in [0, 37, 1024, 2999]:
        for dx in range(16):
            for dy in range(16):
                xs.append(base + dx)
                ys.append(base + dy)
    for e in range(0, 40):
        xs += [n - e, n - e, max(0, n - e - 3)]
        ys += [n - e, max(0, n - e - 5), n - e]
    xs += [n, 0, n]
    ys += [0, n, n]
    for _ in range(300):
        x = int(rng.integers(0, n + 1))
        xs.append(x)
        ys.append(x if rng.random() < 0.7 else int(rng.integers(0, n + 1)))
    return A, B, np.array(xs), np.array(ys)


@pytest.mark.parametrize("method", [0, 1, 2, 7])
@pytest.mark.parametrize("offset", [0, 3, 13])
def test_lcp_methods_match_oracle(ctx, orc, method, offset):
    from paper_2306_17461_gb300 import binding as ed

    rng = np.random.default_rng(10 + method)
    A, B, xs, ys = _lcp_cases(rng)
    # unaligned device bases: views that start `offset` bytes into a buffer
    dA = dev(np.concatenate([np.zeros(offset, np.uint8), A]))[offset:]
    dB = dev(np.concatenate([np.zeros(offset + 5, np.uint8), B]))[offset + 5:]
    got = ed.ed_lcp_dev(ctx.h, dA, dB, xs, ys, method)
    want = np.array([orc.lcp(A, B, int(x), int(y)) for x, y in zip(xs, ys)])
    assert np.array_equal(got, want)


def test_lcp_grid_long_runs(ctx, orc):
    """Runs of hundreds of KiB: the whole-grid slide (chunks, atomicMin),
    with each chunk read by register sweeps (2) or staged in shared memory
    by bulk copies (7), at every alignment of the pair of starts."""
    from paper_2306_17461_gb300 import binding as ed

    rng = np.random.default_rng(3)
    n = 3_000_000
    A = rng.integers(0, 256, n, dtype=np.uint8)
    B = A.copy()
    plant = [123_457, 1_000_003, 1_000_004, 2_999_990]
    for p in plant:
        B[p] ^= 0x5A
    xs = np.array([0, 1, 123_458, 500_000, 1_000_004, 1_000_005, 2_000_000, 2_999_991, 17])
    ys = xs.copy()
    for method in (1, 2, 7, 0):
        got = ed.ed_lcp_dev(ctx.h, dev(A), dev(B), xs, ys, method)
        want = np.array([orc.lcp(A, B, int(x), int(y)) for x, y in zip(xs, ys)])
        assert np.array_equal(got, want), method
    # every (x mod 16, y mod 16) with a mismatch far inside, near a chunk end
    # and at the very end of the strings
    dA, dB = dev(A), dev(B)
    for sx in range(16):
        xs2 = np.array([sx + 16 * k for k in (0, 40_000, 62_500)])
        for sy in range(0, 16, 5):
            ys2 = xs2 - sx + sy
            for method in (2, 7):
                got = ed.ed_lcp_dev(ctx.h, dA, dB, xs2, ys2, method)
                want = np.array([orc.lcp(A, B, int(x), int(y)) for x, y in zip(xs2, ys2)])
                assert np.array_equal(got, want), (method, sx, sy)


@pytest.mark.parametrize("length", [0, 1, 15, 16, 17, 255, 4095, 4096, 4097, 100_003, 1_000_000])
def test_prefix_hash_matches_oracle(ctx, orc, length):
    from paper_2306_17461_gb300 import binding as ed

    rng = np.random.default_rng(length)
    X = rng.integers(0, 256, length, dtype=np.uint8)
    base = ed.ed_hash_base(ctx.h)
    T = ed.ed_prefix_hash_dev(ctx.h, dev(X)).cpu().numpy().view(np.uint64)
    want = orc.prefix_hash(X, base)
    assert np.array_equal(T, want)


def test_prefix_hash_unaligned_and_other_bases(orc):
    from paper_2306_17461_gb300 import binding as ed

    rng = np.random.default_rng(99)
    X = rng.integers(0, 4, 50_001, dtype=np.uint8)
    for seed in [1, 2, 12345]:
        c = ed.Context(device=0, hash_seed=seed)
        base = ed.ed_hash_base(c.h)
        assert 256 <= base < (1 << 61) - 1
        buf = dev(np.concatenate([np.zeros(7, np.uint8), X]))
        T = ed.ed_prefix_hash_dev(c.h, buf[7:]).cpu().numpy().view(np.uint64)
        assert np.array_equal(T, orc.prefix_hash(X, base))
        c.close()


@pytest.mark.parametrize("method", [3, 4])
def test_hash_lcp_matches_direct(ctx, orc, method):
    """Method 3 is the doubling/binary hash search alone, 4 adds the direct
    confirmation; with q = 2^61-1 no collision is expected on these."""
    import torch

    from paper_2306_17461_gb300 import binding as ed

    rng = np.random.default_rng(50 + method)
    A, B, xs, ys = _lcp_cases(rng)
    dA, dB = dev(A), dev(B)
    TA = ed.ed_prefix_hash_dev(ctx.h, dA)
    TB = ed.ed_prefix_hash_dev(ctx.h, dB)
    torch.cuda.synchronize()
    got = ed.ed_lcp_dev(ctx.h, dA, dB, xs, ys, method, TA, TB)
    want = np.array([orc.lcp(A, B, int(x), int(y)) for x, y in zip(xs, ys)])
    assert np.array_equal(got, want)


# ---------------------------------------------------------------- blocked (Sec. 3.3, Alg. 2)
@pytest.mark.parametrize("b", [1, 7, 16, 32, 33, 4096])
@pytest.mark.parametrize("length", [0, 5, 31, 32, 33, 4095, 4097, 100_003])
def test_blocked_prefix_hash_matches_oracle(ctx, orc, b, length):
    """The block prefixes h(X[0..jb)), j = 0..len/b, bit for bit: strides
    that do and do not divide the 16 characters a thread folds or the 4096
    of a scan tile, strings shorter than a block, ragged tails."""
    from paper_2306_17461_gb300 import binding as ed

    rng = np.random.default_rng(1000 * b + length)
    X = rng.integers(0, 256, length, dtype=np.uint8)
    base = ed.ed_hash_base(ctx.h)
    T = ed.ed_prefix_hash_blocked_dev(ctx.h, dev(X), b).cpu().numpy().view(np.uint64)
    assert np.array_equal(T, orc.prefix_hash_blocked(X, b, base))


@pytest.mark.parametrize("method", [5, 6])
def test_blocked_hash_lcp_matches_oracle(orc, method):
    """Methods 5 (search alone) and 6 (confirmed) on blocked tables: equal to
    the oracle's blocked search and to the character LCP."""
    import torch

    from paper_2306_17461_gb300 import binding as ed

    with ed.Context(device=0, hash_block=32) as c:
        rng = np.random.default_rng(70 + method)
        A, B, xs, ys = _lcp_cases(rng)
        dA, dB = dev(A), dev(B)
        TA = ed.ed_prefix_hash_blocked_dev(c.h, dA, 32)
        TB = ed.ed_prefix_hash_blocked_dev(c.h, dB, 32)
        torch.cuda.synchronize()
        got = ed.ed_lcp_dev(c.h, dA, dB, xs, ys, method, TA, TB)
        base = ed.ed_hash_base(c.h)
        hA, hB = TA.cpu().numpy().view(np.uint64), TB.cpu().numpy().view(np.uint64)
        want = np.array([orc.lcp(A, B, int(x), int(y)) for x, y in zip(xs, ys)])
        if method == 5:
            ob = np.array([orc.hash_lcp_blocked(A, hA, B, hB, 32, base, int(x), int(y)) for x, y in zip(xs, ys)])
            assert np.array_equal(ob, want)  # no collision on these inputs
        assert np.array_equal(got, want)


@pytest.mark.parametrize("blocked", [False, True])
def test_confirmation_makes_wrong_hash_answers_exact(orc, blocked):
    """The safety net for hash collisions (Sec. 2 remark): every hash answer
    is confirmed by a direct compare.  Tables of A and B built with two
    different bases disagree on equal substrings, so the hash search alone
    answers wrongly on most queries; confirmed, every answer is the
    character LCP."""
    import torch

    from paper_2306_17461_gb300 import binding as ed

    rng = np.random.default_rng(77 + blocked)
    A, B, xs, ys = _lcp_cases(rng)
    dA, dB = dev(A), dev(B)
    with ed.Context(device=0, hash_seed=1, hash_block=32) as c1, ed.Context(device=0, hash_seed=2) as c2:
        if blocked:
            TA = ed.ed_prefix_hash_blocked_dev(c1.h, dA, 32)
            TB = ed.ed_prefix_hash_blocked_dev(c2.h, dB, 32)
            alone, confirmed = 5, 6
        else:
            TA = ed.ed_prefix_hash_dev(c1.h, dA)
            TB = ed.ed_prefix_hash_dev(c2.h, dB)
            alone, confirmed = 3, 4
        torch.cuda.synchronize()
        want = np.array([orc.lcp(A, B, int(x), int(y)) for x, y in zip(xs, ys)])
        wrong = ed.ed_lcp_dev(c1.h, dA, dB, xs, ys, alone, TA, TB)
        reach = want >= 8  # queries the leading direct window does not settle
        assert reach.sum() > 20 and (wrong[reach] != want[reach]).mean() > 0.5  # the tables disagree
        got = ed.ed_lcp_dev(c1.h, dA, dB, xs, ys, confirmed, TA, TB)
        assert np.array_equal(got, want)

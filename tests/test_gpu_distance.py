"""The single-pair path (one persistent launch of Algorithm 1) against the
oracle: frontiers round by round, distances on random, planted and
degenerate pairs, every phase of the kernel (narrow CTA, wide grid, long
slides handed to the grid, hash LCP), host and device entry points.
Integer results: the tolerance is zero."""
import numpy as np
import pytest

from gpu_util import dev, mirror_oracle_frontier
from paper_2306_17461_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# kernel configurations exercised: default (32 rounds per block); 16 and
# 64 rounds per block (the largest), the latter with tiles as narrow as
# allowed; narrow first tiles (many epoch changes, the band crosses many
# tiles); one round per block; odd block lengths and few CTAs; one CTA; the
# hash LCP on full and on blocked prefix tables (Sec. 3.3; blocks of 32 and
# of 7 characters)
CONFIGS = {
    "default": {},
    "h16": {"block_rounds": 16},
    "h64_narrow": {"block_rounds": 64, "tile_width": 1},
    "wide": {"tile_width": 1, "block_rounds": 4},
    "wide_g3": {"tile_width": 2, "grid_ctas": 3, "block_rounds": 3},
    "h1": {"block_rounds": 1, "tile_width": 1},
    "one_cta": {"grid_ctas": 1},
    "hash": {"lcp_mode": 2},
    "hash_wide": {"lcp_mode": 2, "tile_width": 1, "block_rounds": 5},
    "bhash": {"lcp_mode": 3},
    "bhash_b7_wide": {"lcp_mode": 3, "hash_block": 7, "tile_width": 1, "block_rounds": 5},
    # long slides: the CTA scans 4 chunks alone first, half the CTAs serve
    # slides, a warp hands a slide on after 1 KiB; and no helper CTAs at all
    "slides_lc4_h2": {"local_chunks": 4, "help_div": 2, "warp_cap": 1024},
    "no_helpers": {"help_div": -1, "local_chunks": -1},
}


@pytest.fixture(scope="module")
def ctxs():
    from paper_2306_17461_gb300 import binding as ed

    cs = {name: ed.Context(device=0, **cfg) for name, cfg in CONFIGS.items()}
    yield cs
    for c in cs.values():
        c.close()


@pytest.mark.parametrize("cfg", list(CONFIGS))
def test_frontiers_match_oracle(ctxs, orc, cfg):
    from paper_2306_17461_gb300 import binding as ed

    ctx = ctxs[cfg]
    rng = np.random.default_rng(21)
    for trial in range(12):
        n = int(rng.integers(0, 300))
        sigma = [2, 4, 256][trial % 3]
        A, B = W.random_pair(rng, n, int(rng.integers(0, 25)), sigma)
        k = orc.lv(A, B)
        T = k + 2
        kg, F = ed.ed_frontiers_dev(ctx.h, dev(A), dev(B), T)
        ko, Fo = orc.lv_frontiers(A, B, T)
        assert kg == ko == k
        G = mirror_oracle_frontier(Fo, T, orc.NEG, ed.NEG32)
        assert np.array_equal(F.astype(np.int64), G), (cfg, trial)


@pytest.mark.parametrize("cfg", list(CONFIGS))
def test_random_pairs(ctxs, orc, cfg):
    ctx = ctxs[cfg]
    rng = np.random.default_rng(7)
    for trial in range(25):
        sigma = [2, 4, 64, 256][trial % 4]
        n = int(rng.integers(0, 20000))
        k = int(rng.integers(0, max(1, n // 10) + 1))
        A, B = W.random_pair(rng, n, k, sigma)
        assert ctx.distance_dev(dev(A), dev(B)) == orc.lv(A, B), (cfg, trial)


@pytest.mark.parametrize("cfg", ["default", "wide", "hash"])
def test_degenerate_cases(ctxs, orc, cfg):
    ctx = ctxs[cfg]
    E = np.zeros(0, np.uint8)
    cases = [
        (E, E),
        (E, np.arange(7, dtype=np.uint8)),
        (np.arange(9, dtype=np.uint8), E),
        (np.zeros(1000, np.uint8), np.zeros(1000, np.uint8)),  # identical, all one symbol
        (np.zeros(1000, np.uint8), np.ones(1000, np.uint8)),   # nothing matches
        (np.zeros(500, np.uint8), np.zeros(1500, np.uint8)),   # runs of one symbol: long slides everywhere
        (np.array([0, 0, 1], np.uint8), np.array([0, 1], np.uint8)),  # NUL bytes
        (np.arange(256, dtype=np.uint8), np.arange(255, -1, -1, dtype=np.uint8)),
        (np.array([5], np.uint8), np.array([5], np.uint8)),
        (np.array([5], np.uint8), np.array([6], np.uint8)),
    ]
    for A, B in cases:
        want = orc.dp(A, B) if A.size * B.size <= 4_000_000 else orc.lv(A, B)
        assert ctx.distance_dev(dev(A), dev(B)) == want
        assert ctx.distance(A, B) == want


def test_unaligned_device_strings(ctxs, orc):
    ctx = ctxs["default"]
    p = W.make_pair(31, 100_000, 60, sigma=4)
    want = orc.lv(p.A, p.B)
    for oa, ob in [(1, 2), (3, 15), (8, 0), (15, 7)]:
        bufA = dev(np.concatenate([np.full(oa, 9, np.uint8), p.A]))
        bufB = dev(np.concatenate([np.full(ob, 9, np.uint8), p.B]))
        assert ctx.distance_dev(bufA[oa:], bufB[ob:]) == want


@pytest.mark.parametrize("cfg", list(CONFIGS))
def test_long_slides(ctxs, orc, cfg):
    """Few edits far apart: slides of up to megabytes, which go from one
    thread to one warp to the whole grid."""
    ctx = ctxs[cfg]
    for idx, (n, k) in enumerate([(2_000_000, 1), (2_000_000, 3), (3_000_000, 12), (500_000, 0)]):
        p = W.make_pair(40 + idx, n, k, sigma=256)
        want = orc.lv(p.A, p.B)
        assert ctx.distance_dev(dev(p.A), dev(p.B)) == want, (cfg, n, k)
        st = ctx.stats()
        assert st["k"] == want
        if cfg == "default" and k > 0:
            assert st["long_slides"] >= 1


def test_stats_counters(ctxs, orc):
    ctx = ctxs["default"]
    p = W.make_pair(55, 300_000, 400, sigma=4)
    k, rounds, ext = orc.lv(p.A, p.B, with_stats=True)
    assert ctx.distance_dev(dev(p.A), dev(p.B)) == k
    st = ctx.stats()
    assert st["extensions"] == ext
    assert st["kernel_launches"] == 1
    assert st["compared_bytes"] >= 2 * (p.A.size - p.edits)


@pytest.mark.parametrize("k", [10, 1000, 10_000])
def test_mid_workload_reduced(ctxs, orc, k):
    """The n = 10^8 alphabet-4 workload, reduced to n = 10^7."""
    p = W.single_mid(k, n=10_000_000)
    want = orc.lv(p.A, p.B, nthreads=8)
    for cfg in ["default", "hash"]:
        assert ctxs[cfg].distance_dev(dev(p.A), dev(p.B)) == want, cfg


def test_single_small_full_size(ctxs, orc):
    """The n = 10^6, 100 planted edits workload at full size."""
    p = W.single_small()
    want = orc.lv(p.A, p.B)
    assert want <= 100
    for cfg in ["default", "wide", "hash"]:
        assert ctxs[cfg].distance_dev(dev(p.A), dev(p.B)) == want
        assert ctxs[cfg].distance(p.A, p.B) == want


def test_large_workload_reduced(ctxs, orc):
    """The Zipf(1.1), bursty workload, reduced to n = 2*10^7, 2000 edits."""
    p = W.single_large(n=20_000_000, k=2000)
    want = orc.lv(p.A, p.B, nthreads=8)
    assert ctxs["default"].distance_dev(dev(p.A), dev(p.B)) == want


def test_round_cap_is_reported():
    """A pair needing more rounds than max_rounds ends with ED_ELIMIT, and
    the context stays usable for the next pair."""
    from paper_2306_17461_gb300 import binding as ed

    p = W.make_pair(95, 20_000, 300, sigma=4)
    with ed.Context(device=0, max_rounds=64) as c:
        with pytest.raises(ed.EdError) as e:
            ed.ed_distance_dev(c.h, dev(p.A), dev(p.B))
        assert e.value.code == ed.ED_ELIMIT
        q = W.make_pair(96, 20_000, 20, sigma=4)
        assert ed.ed_distance_dev(c.h, dev(q.A), dev(q.B)) <= 20


def test_band_outgrows_tiles_and_resumes(orc):
    """A single pair starts on narrow tiles (2048 diagonals per CTA).  When
    its band outgrows them, the group saves the band frontier and the host
    resumes from that round on tiles four times wider.  On one CTA, a pair
    at k ~ 6000 resumes twice (2048 -> 8192 -> 16384); the distance is the
    oracle's and no round is recomputed."""
    from paper_2306_17461_gb300 import binding as ed

    p = W.make_pair(120, 100_000, 6000, sigma=4)
    want = orc.lv(p.A, p.B)
    assert want > 4096  # the band (2k + 1 diagonals) passes 8192
    with ed.Context(device=0, grid_ctas=1) as c:
        assert ed.ed_distance_dev(c.h, dev(p.A), dev(p.B)) == want
        st = c.stats()
        assert st["kernel_launches"] == 3
        # every round counted once: a resumed launch starts where the last stopped
        assert st["extensions"] == orc.lv(p.A, p.B, with_stats=True)[2]


@pytest.mark.parametrize("p0", [0.5, 0.9, 0.99])
def test_lcp_length_workload_reduced(ctxs, orc, p0):
    """Fig. 4's inputs (two skewed symbols, long chance matches) at n = 2e5:
    every LCP mode gives the oracle's distance."""
    from paper_2306_17461_gb300 import binding as ed

    for k in (300, 1000):
        p = W.lcp_length_pair(k, p0, n=200_000)
        want = orc.lv(p.A, p.B)
        for cfg in ("default", "hash", "bhash"):
            assert ctxs[cfg].distance_dev(dev(p.A), dev(p.B)) == want, (cfg, k, p0)


def test_skew_lengthens_the_slides(ctxs):
    """Fig. 4's x axis: the mean LCP per diagonal-extension grows with the
    skew of the two symbols.  (Between P(0) = 0.5 and 0.9 the exact mean
    differs by a few per cent only, about what CTAs that run blocks past k
    add to the device's count; 0.99 and 0.999 are well apart.)"""
    means = []
    for p0 in (0.5, 0.99, 0.999):
        p = W.lcp_length_pair(1000, p0, n=200_000)
        ctxs["default"].distance_dev(dev(p.A), dev(p.B))
        st = ctxs["default"].stats()
        means.append(st["slide_chars"] / st["extensions"])
    assert means[0] < means[1] < means[2], means

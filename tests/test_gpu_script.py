"""Edit scripts traced back from the kernel's frontiers: valid (they turn A
into B with matching characters between operations) and as long as the
oracle's distance, hence optimal; on random, planted and degenerate pairs
and under several tilings of the kernel.  Scripts are not unique, so
only validity and length are compared."""
import numpy as np
import pytest

from gpu_util import dev
from paper_2306_17461_gb300 import workloads as W
from script_check import script_transforms

pytestmark = pytest.mark.gpu

CONFIGS = {"default": {}, "wide": {"tile_width": 1, "block_rounds": 4}, "one_cta": {"grid_ctas": 1}}


@pytest.fixture(scope="module")
def ctxs():
    from paper_2306_17461_gb300 import binding as ed

    cs = {name: ed.Context(device=0, **cfg) for name, cfg in CONFIGS.items()}
    yield cs
    for c in cs.values():
        c.close()


def _check(ctx, orc, A, B, slack=3):
    from paper_2306_17461_gb300 import binding as ed

    k = orc.lv(A, B)
    kg, ops = ed.ed_edit_script_dev(ctx.h, dev(A), dev(B), k + slack)
    assert kg == k
    assert len(ops) == k
    assert script_transforms(A, B, ops)


@pytest.mark.parametrize("cfg", list(CONFIGS))
def test_random_and_planted_pairs(ctxs, orc, cfg):
    rng = np.random.default_rng(5)
    for trial in range(16):
        sigma = [2, 4, 256][trial % 3]
        n = int(rng.integers(0, 2000))
        A, B = W.random_pair(rng, n, int(rng.integers(0, 120)), sigma)
        _check(ctxs[cfg], orc, A, B)


def test_degenerate_pairs(ctxs, orc):
    ctx = ctxs["default"]
    rng = np.random.default_rng(6)
    x = rng.integers(0, 4, 300, dtype=np.uint8)
    empty = np.zeros(0, np.uint8)
    _check(ctx, orc, x, x)                                       # k = 0
    _check(ctx, orc, x, empty)                                   # deletions only
    _check(ctx, orc, empty, x[:200])                             # insertions only
    _check(ctx, orc, x[:150], x[:150] + 4)                       # disjoint alphabets
    _check(ctx, orc, x, np.concatenate([x[:100], x[180:]]))      # one long deletion
    _check(ctx, orc, np.zeros(500, np.uint8), np.zeros(350, np.uint8))  # runs


def test_long_pair_near_the_bound(ctxs, orc):
    # n = 10^6 with about 3000 planted edits: frontiers of ~3000 rounds
    p = W.make_pair(31, 1_000_000, 3000, sigma=4)
    _check(ctxs["default"], orc, p.A, p.B, slack=1)


def test_distance_past_the_frontier_dump_bound(ctxs, orc):
    # k ~ 6000: past the 4096 rounds of ed_frontiers_dev, within the script's bound
    p = W.make_pair(34, 2_000_000, 6000, sigma=4)
    _check(ctxs["default"], orc, p.A, p.B, slack=1)


def test_distance_past_the_bound_is_reported(ctxs, orc):
    from paper_2306_17461_gb300 import binding as ed

    p = W.make_pair(32, 20_000, 300, sigma=4)
    k = orc.lv(p.A, p.B)
    with pytest.raises(ed.EdError) as e:
        ed.ed_edit_script_dev(ctxs["default"].h, dev(p.A), dev(p.B), k - 1)
    assert e.value.code == ed.ED_ELIMIT

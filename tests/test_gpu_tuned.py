"""The tuning table's choices on the GPU: for pairs of every length and
edit-rate class the committed table covers, a context that takes its launch
parameters from the table (ed_config.tune, with the pair's expected distance
as the hint) computes the oracle's distance; and the parameters it would
choose are the ones ed_tune_lookup reports."""
import os

import pytest

from gpu_util import dev
from paper_2306_17461_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TABLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2306_17461_gb300",
                     "tune_table.tsv")


@pytest.mark.skipif(not os.path.exists(TABLE), reason="no committed table")
@pytest.mark.parametrize("n,k", [(200_000, 1), (200_000, 50), (1_000_000, 1000), (4_000_000, 30), (4_000_000, 4000),
                                  (40_000_000, 40)])
def test_tuned_contexts_match_oracle(orc, n, k):
    from paper_2306_17461_gb300 import binding as ed

    p = W.make_pair(120, n, k, sigma=4, extra=k)
    want = orc.lv(p.A, p.B, nthreads=8)
    row = ed.ed_tune_lookup(n, n, k, TABLE)
    with ed.Context(device=0, tune=1, distance_hint=k) as c:
        assert c.distance_dev(dev(p.A), dev(p.B)) == want
        assert c.distance(p.A, p.B) == want
    # the same parameters set explicitly give the same distance
    with ed.Context(device=0, lcp_mode=row.lcp_mode, block_rounds=row.block_rounds, tile_width=row.tile_width,
                    warp_cap=row.warp_cap, local_chunks=row.local_chunks, help_div=row.help_div) as c:
        assert c.distance_dev(dev(p.A), dev(p.B)) == want

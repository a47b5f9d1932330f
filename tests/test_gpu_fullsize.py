"""Full-size workloads, in the launch configuration the benchmark times (the
tuning table's row for the pair) and in the built-in defaults, against the
oracle (exact: the distance is an integer).

* n = 10^8, alphabet 4, k planted in {10, 10^3, 10^5}: the oracle runs
  Algorithm 1 whole (OpenMP over the diagonals of a round for 10^5);
* n = 10^9, Zipf(1.1), 10^4 bursty edits: the oracle runs whole;
* the serving and batch paths are covered at reduced size elsewhere.
"""
import os

import pytest

from gpu_util import dev
from paper_2306_17461_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2306_17461_gb300 import binding as ed

    c = ed.Context(device=0)
    yield c
    c.close()


def bench_ctx(p):
    """The context the benchmark times the pair on: launch parameters from
    the tuning table, the planted edit count as the expected distance."""
    from paper_2306_17461_gb300 import binding as ed

    return ed.Context(device=0, tune=1, distance_hint=int(p.edits))


@pytest.mark.parametrize("k", [10, 1000, 100_000])
def test_mid_full_size(ctx, orc, k):
    p = W.single_mid(k)
    want = orc.lv(p.A, p.B, nthreads=os.cpu_count() or 1)
    dA, dB = dev(p.A), dev(p.B)
    tc = bench_ctx(p)
    try:
        assert tc.distance_dev(dA, dB) == want
        st = tc.stats()
        assert st["k"] == want and st["extensions"] > 0
    finally:
        tc.close()
    # the built-in defaults, and end to end through host buffers as well
    assert ctx.distance_dev(dA, dB) == want
    if k == 1000:
        assert ctx.distance(p.A, p.B) == want


def test_large_full_size(ctx, orc):
    p = W.single_large()
    want = orc.lv(p.A, p.B, nthreads=os.cpu_count() or 1)
    assert abs(p.A.size - p.B.size) <= want <= p.edits
    dA, dB = dev(p.A), dev(p.B)
    tc = bench_ctx(p)
    try:
        assert tc.distance_dev(dA, dB) == want
    finally:
        tc.close()
    assert ctx.distance_dev(dA, dB) == want

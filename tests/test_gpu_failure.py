"""Failure detection without a GPU fault: every device-side wait of the
tile kernel is bounded by %globaltimer.  With a bound of 1 ns the first
poll of a neighbour's flag gives up: the kernel records where, every CTA
leaves, and the host returns ED_ETIMEOUT with the record; the device stays
usable and a context with the default bound computes the exact distance
on the same strings."""
import pytest

from gpu_util import dev
from paper_2306_17461_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.timeout(300)
def test_bounded_wait_gives_up_and_the_device_stays_usable(orc):
    from paper_2306_17461_gb300 import binding as ed

    # thousands of rounds over the whole grid: neighbour waits every block
    p = W.make_pair(51, 1_000_000, 3000, sigma=4)
    want = orc.lv(p.A, p.B)
    dA, dB = dev(p.A), dev(p.B)
    c = ed.Context(device=0, spin_limit_ns=1)
    try:
        try:
            k = c.distance_dev(dA, dB)
            assert k == want  # no wait outlived its first poll (unlikely)
        except ed.EdError as e:
            assert e.code == ed.ED_ETIMEOUT, str(e)
    finally:
        c.close()
    c2 = ed.Context(device=0)
    try:
        assert c2.distance_dev(dA, dB) == want
    finally:
        c2.close()

"""Failure detection without a GPU fault.

* Every device-side wait of the tile kernel is bounded by %globaltimer.
  With a bound of 1 ns a wait that cannot be answered at once gives up: the
  kernel records where (site, CTA, round), every CTA leaves, and the host
  returns ED_ETIMEOUT with that record.  The pair used makes such a wait
  certain: tiles beyond the band skip ahead and then wait for their inner
  neighbour to compute about a thousand rounds.  The device stays usable: a
  context with the default bound computes the exact distance on the same
  strings.
* Host-side refusals: a memory budget too small for the strings returns
  ED_ENOMEM before anything is allocated, and serving refuses admission
  (ED_EBUSY) when the arena cannot hold a request while another one is
  resident, then admits it once that one has retired."""
import re
import time

import pytest

from gpu_util import dev
from paper_2306_17461_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.timeout(300)
def test_bounded_wait_gives_up_and_the_device_stays_usable(orc):
    from paper_2306_17461_gb300 import binding as ed

    # thousands of rounds over the whole grid
    p = W.make_pair(51, 1_000_000, 3000, sigma=4)
    want = orc.lv(p.A, p.B)
    dA, dB = dev(p.A), dev(p.B)
    c = ed.Context(device=0, spin_limit_ns=1)
    try:
        with pytest.raises(ed.EdError) as ei:
            c.distance_dev(dA, dB)
        assert ei.value.code == ed.ED_ETIMEOUT, str(ei.value)
        m = re.search(r"kernel check failed: site (\d+) cta (\d+) t (\d+)", str(ei.value))
        assert m, str(ei.value)
        # 1 job close, 2 group barrier, 3 idle CTA, 4 neighbours' edge words, 5 epoch barrier
        assert 1 <= int(m.group(1)) <= 5
    finally:
        c.close()
    c2 = ed.Context(device=0)
    try:
        assert c2.distance_dev(dA, dB) == want
    finally:
        c2.close()


def test_budget_too_small_for_the_strings():
    import numpy as np

    from paper_2306_17461_gb300 import binding as ed

    c = ed.Context(device=0, mem_budget_bytes=1 << 20)
    try:
        A = np.zeros(2 << 20, np.uint8)
        with pytest.raises(ed.EdError) as ei:
            c.distance(A, A)
        assert ei.value.code == ed.ED_ENOMEM
    finally:
        c.close()


@pytest.mark.timeout(300)
def test_serving_refuses_admission_on_memory_then_admits(orc):
    from paper_2306_17461_gb300 import binding as ed

    # arena: half of a 200 MB budget; a resident 2 x 30 MB pair leaves no room
    # for a second one
    big = W.make_pair(52, 30_000_000, 30_000, sigma=4)
    small = W.make_pair(53, 30_000_000, 10, sigma=4)
    want_big, want_small = orc.lv(big.A, big.B, nthreads=8), orc.lv(small.A, small.B)
    c = ed.Context(device=0, mem_budget_bytes=200 << 20, max_inflight=64)
    try:
        t1 = ed.ed_submit(c.h, big.A, big.B)
        with pytest.raises(ed.EdError) as ei:
            ed.ed_submit(c.h, small.A, small.B)
        assert ei.value.code == ed.ED_EBUSY
        # admitted once the first request has retired and freed its memory
        t2 = None
        k1 = None
        deadline = time.time() + 240
        while t2 is None and time.time() < deadline:
            st, k = ed.ed_poll(c.h, t1)
            if st == ed.ED_OK:
                k1 = k
            try:
                t2 = ed.ed_submit(c.h, small.A, small.B)
            except ed.EdError as e:
                assert e.code == ed.ED_EBUSY
                time.sleep(0.01)
        assert t2 is not None
        while k1 is None:
            st, k = ed.ed_poll(c.h, t1)
            if st == ed.ED_OK:
                k1 = k
            time.sleep(0.002)
        while True:
            st, k2 = ed.ed_poll(c.h, t2)
            if st == ed.ED_OK:
                break
            time.sleep(0.002)
        assert (k1, k2) == (want_big, want_small)
        assert ed.ed_serve_counters(c.h)["admitted"] == 2
    finally:
        c.close()

"""Full-size parity of the batched and served workloads against the
oracle's cached distances (tests/golden/*_distances.tsv, written by a
script that calls only the oracle): all 4096 batched pairs (n log-uniform
on [10^3, 10^6]) in one batched call, and all 512 served pairs (n
log-uniform on [10^2, 10^7], edit rates up to 10%) submitted together and
served concurrently, with a sample of them served alone as well.  Integer
results: equal element by element."""
import time

import numpy as np
import pytest

import fullsize_cache as FC
from paper_2306_17461_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


@pytest.mark.timeout(900)
def test_batch_4096_pairs_full_size():
    from paper_2306_17461_gb300 import binding as ed

    cache = FC.load("batch")
    assert FC.complete("batch")
    pairs = W.batch_pairs(4096)
    want = np.array([cache[i][3] for i in range(4096)])
    c = ed.Context(device=0)
    try:
        got = ed.ed_distance_batch_dev(c.h, [_dev(p.A) for p in pairs], [_dev(p.B) for p in pairs])
    finally:
        c.close()
    assert np.array_equal(got, want)


def _serve(c, pairs, timeout_s):
    from paper_2306_17461_gb300 import binding as ed

    tickets = {}
    got = {}
    i = 0
    t0 = time.time()
    while i < len(pairs) or tickets:
        while i < len(pairs):
            try:
                tickets[ed.ed_submit(c.h, pairs[i].A, pairs[i].B)] = i
                i += 1
            except ed.EdError as e:
                if e.code != ed.ED_EBUSY:
                    raise
                break
        for t in list(tickets):
            st, k = ed.ed_poll(c.h, t)
            if st == ed.ED_OK:
                got[tickets.pop(t)] = k
        assert time.time() - t0 < timeout_s, "serving did not finish"
        time.sleep(0.001)
    return np.array([got[j] for j in range(len(pairs))])


@pytest.mark.timeout(1800)
def test_serve_512_pairs_full_size_mixed_and_alone():
    from paper_2306_17461_gb300 import binding as ed

    if not FC.complete("serve"):
        pytest.skip("the oracle's cache of the served set is incomplete")
    cache = FC.load("serve")
    pairs = W.serve_pairs(512)
    want = np.array([cache[i][3] for i in range(512)])
    c = ed.Context(device=0, max_inflight=1024)
    try:
        mixed = _serve(c, pairs, 1500)
        assert np.array_equal(mixed, want)
        # alone: the smallest, a median one, and the largest by work
        order = sorted(range(512), key=lambda i: cache[i][3] ** 2 + cache[i][0])
        for i in (order[0], order[256], order[-1]):
            alone = _serve(c, [pairs[i]], 600)
            assert alone[0] == mixed[i] == want[i]
    finally:
        c.close()

"""Batched and served pairs against the oracle (bit-exact): the persistent
work-queue kernel, pairs whose band outgrows one CTA, host and device entry
points, and continuous batching (admission, resident frontiers, retirement)
with the same result alone and in a mix."""
import time

import numpy as np
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


def _pairs_reduced(npairs=384, n_hi=1e5):
    return W.batch_pairs(npairs, n_lo=1e3, n_hi=n_hi)


def test_batch_dev_matches_oracle(ctx, orc):
    from paper_2306_17461_gb300 import binding as ed

    pairs = _pairs_reduced()
    # a few pairs whose band outgrows one CTA (k > 2048)
    for i in range(4):
        pairs.append(W.make_pair(60 + i, 30_000, 5000, sigma=4))
    pairs.append(W.make_pair(70, 0, 0))
    pairs.append(W.Pair(np.zeros(0, np.uint8), np.arange(10, dtype=np.uint8), 10, "empty A"))
    want = orc.many("lv", [(p.A, p.B) for p in pairs])
    dA = [dev(p.A) for p in pairs]
    dB = [dev(p.B) for p in pairs]
    got = ed.ed_distance_batch_dev(ctx.h, dA, dB)
    assert np.array_equal(got, want)
    st = ctx.stats()
    assert st["extensions"] > 0


def _tail_burst_pair(n=200_000, k=16_000, tail=40_000, extra=0):
    """Edits only in the last `tail` characters: the frontier runs far ahead
    in the first rounds, so an estimate of the distance from early progress
    is far too low."""
    rng = W.rng_for(81, extra)
    sym = W.Symbols(4)
    A = sym.draw(rng, n)
    pos = np.sort(rng.choice(np.arange(n - tail, n), size=k, replace=False))
    return W.Pair(A, W.plant(rng, A, pos, sym), k, "tail burst")


def test_batch_band_outgrows_estimated_group(orc):
    """A parked pair placed on a group too small for its band ends with the
    per-pair 'too wide' status and runs again on a larger group (one more
    tile launch); every distance still equals the oracle's."""
    from paper_2306_17461_gb300 import binding as ed

    c = ed.Context(device=0, grid_ctas=4)
    try:
        pairs = [W.make_pair(90 + i, 40_000, 2500, sigma=4) for i in range(2)]
        pairs.append(_tail_burst_pair())
        want = orc.many("lv", [(p.A, p.B) for p in pairs])
        assert want[2] > 8192  # wider than one CTA's tiles hold
        got = ed.ed_distance_batch_dev(c.h, [dev(p.A) for p in pairs], [dev(p.B) for p in pairs])
        assert np.array_equal(got, want)
        # the batch launch, the tile launch, and the retry of the wide pair
        assert c.stats()["kernel_launches"] == 3
    finally:
        c.close()


def test_batch_host_matches_oracle(ctx, orc):
    from paper_2306_17461_gb300 import binding as ed

    pairs = _pairs_reduced(128, 3e4)
    want = orc.many("lv", [(p.A, p.B) for p in pairs])
    got = ed.ed_distance_batch(ctx.h, [p.A for p in pairs], [p.B for p in pairs])
    assert np.array_equal(got, want)


def _serve_all(ctx, pairs, timeout_s=120.0):
    from paper_2306_17461_gb300 import binding as ed

    tickets = []
    for p in pairs:
        while True:
            try:
                tickets.append(ed.ed_submit(ctx.h, p.A, p.B))
                break
            except ed.EdError as e:
                if e.code != ed.ED_EBUSY:
                    raise
                time.sleep(0.001)
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for i, t in enumerate(tickets):
            if i in out:
                continue
            st, k = ed.ed_poll(ctx.h, t)
            if st == ed.ED_OK:
                out[i] = k
        assert time.time() - t0 < timeout_s, "serving did not finish"
        time.sleep(0.0005)
    return np.array([out[i] for i in range(len(tickets))])


def test_serving_matches_oracle_alone_and_mixed(orc):
    from paper_2306_17461_gb300 import binding as ed

    c = ed.Context(device=0, max_inflight=64)
    pairs = W.serve_pairs(96, n_lo=1e2, n_hi=2e5)
    want = orc.many("lv", [(p.A, p.B) for p in pairs])
    mixed = _serve_all(c, pairs)
    assert np.array_equal(mixed, want)
    # each pair alone gives the same answer as in the mix
    for i in [0, 5, 17, 42]:
        alone = _serve_all(c, [pairs[i]])
        assert alone[0] == mixed[i] == want[i]
    cnt = ed.ed_serve_counters(c.h)
    assert cnt["admitted"] == cnt["completed"] == len(pairs) + 4
    assert cnt["inflight"] == 0
    c.close()


def test_serving_time_slices_wide_pairs(orc):
    """Pairs whose band outgrows one CTA run on the tile kernel a slice per
    engine step, their band frontiers saved and resumed between steps.
    Small pairs submitted after a long pair finish before it, and every
    result is exact: the long pair has disjoint alphabets (no character
    matches, so the distance is max(n, m) after that many rounds), the
    others are checked against the oracle."""
    from paper_2306_17461_gb300 import binding as ed

    rng = np.random.default_rng(99)
    n_long = 100_000
    long_pair = (rng.integers(0, 4, n_long, dtype=np.uint8), rng.integers(4, 8, n_long, dtype=np.uint8))
    heavy = W.make_pair(97, 500_000, 25_000, sigma=4)
    small = [W.make_pair(98, 10_000, 10, sigma=4, extra=i) for i in range(16)]
    want = [n_long] + list(orc.many("lv", [(p.A, p.B) for p in [heavy] + small]))
    c = ed.Context(device=0, max_inflight=64)
    try:
        tickets = [ed.ed_submit(c.h, *long_pair), ed.ed_submit(c.h, heavy.A, heavy.B)]
        time.sleep(0.02)  # the long pairs are on the device before the rest arrive
        tickets += [ed.ed_submit(c.h, p.A, p.B) for p in small]
        got, order = {}, []
        t0 = time.time()
        while len(got) < len(tickets):
            for i, t in enumerate(tickets):
                if i not in got:
                    st, k = ed.ed_poll(c.h, t)
                    if st == ed.ED_OK:
                        got[i] = k
                        order.append(i)
            assert time.time() - t0 < 120, "serving did not finish"
            time.sleep(0.0005)
        assert [got[i] for i in range(len(tickets))] == want
        # the small pairs did not wait for the long one
        assert order.index(0) > max(order.index(i) for i in range(2, len(tickets)))
        assert ed.ed_serve_counters(c.h)["slices"] >= 1
    finally:
        c.close()


def test_poll_unknown_ticket(ctx):
    from paper_2306_17461_gb300 import binding as ed

    with pytest.raises(ed.EdError) as e:
        ed.ed_poll(ctx.h, 987654321)
    assert e.value.code == ed.ED_ENOTFOUND


def test_admission_refuses_when_slots_full(orc):
    from paper_2306_17461_gb300 import binding as ed

    c = ed.Context(device=0, max_inflight=2)
    big = W.make_pair(80, 2_000_000, 3000, sigma=4)
    t1 = ed.ed_submit(c.h, big.A, big.B)
    t2 = ed.ed_submit(c.h, big.A, big.B)
    refused = False
    try:
        ed.ed_submit(c.h, big.A, big.B)
    except ed.EdError as e:
        refused = e.code == ed.ED_EBUSY
    # the third may have been admitted only if one of the first two finished
    cnt = ed.ed_serve_counters(c.h)
    assert refused or cnt["completed"] >= 1
    want = orc.lv(big.A, big.B)
    res = []
    for t in (t1, t2):
        while True:
            st, k = ed.ed_poll(c.h, t)
            if st == ed.ED_OK:
                res.append(k)
                break
            time.sleep(0.001)
    assert res == [want, want]
    c.close()


def test_submit_dev_strings_written_on_a_side_stream(orc):
    """ed_submit_dev: device strings that a copy on the caller's side stream
    is still writing when they are submitted; the engine waits for that
    stream's work.  Mixed with host-submitted pairs; every result equals the
    oracle's."""
    import torch

    from paper_2306_17461_gb300 import binding as ed

    c = ed.Context(device=0, max_inflight=64)
    try:
        pairs = [W.make_pair(110, 3_000_000, 40, sigma=4, extra=i) for i in range(4)]
        pairs += [W.make_pair(111, 300_000, 9000, sigma=4)]  # wider than one CTA's band
        want = orc.many("lv", [(p.A, p.B) for p in pairs])
        side = torch.cuda.Stream()
        bufs, tickets = [], []
        for i, p in enumerate(pairs):
            hA = torch.from_numpy(p.A).pin_memory()
            hB = torch.from_numpy(p.B).pin_memory()
            with torch.cuda.stream(side):
                dA = torch.empty(p.A.size, dtype=torch.uint8, device="cuda")
                dB = torch.empty(p.B.size, dtype=torch.uint8, device="cuda")
                dA.copy_(hA, non_blocking=True)
                dB.copy_(hB, non_blocking=True)
            bufs.append((dA, dB, hA, hB))
            if i % 2:
                tickets.append(ed.ed_submit(c.h, p.A, p.B))
            else:
                tickets.append(ed.ed_submit_dev(c.h, dA, dB, stream=side))
        got = {}
        t0 = time.time()
        while len(got) < len(tickets):
            for i, t in enumerate(tickets):
                if i not in got:
                    st, k = ed.ed_poll(c.h, t)
                    if st == ed.ED_OK:
                        got[i] = k
            assert time.time() - t0 < 120, "serving did not finish"
            time.sleep(0.0005)
        assert [got[i] for i in range(len(tickets))] == list(want)
        # bad arguments: a null string with a length
        lib = ed.load()
        import ctypes

        tk = ctypes.c_uint64()
        assert lib.ed_submit_dev(c.h, None, 5, None, 0, ctypes.byref(tk), None) == ed.ED_EINVAL
    finally:
        c.close()

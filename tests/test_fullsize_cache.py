"""The cached oracle distances of the full-size batched and served pair sets
against the generators and the oracle itself (CPU only): every entry
describes the pair its index generates (lengths, planted edits), obeys the
distance bounds |n - m| <= k <= planted, and the smallest pairs of each set,
recomputed here by the oracle (Algorithm 1) and by the DP of Sec. 1, give
the cached value."""
import numpy as np
import pytest

import fullsize_cache as FC
from paper_2306_17461_gb300 import workloads as W


@pytest.mark.parametrize("name", ["batch", "serve"])
def test_cache_matches_generators_and_bounds(name):
    cache = FC.load(name)
    npairs = FC.FILES[name][1]
    assert set(cache) <= set(range(npairs))
    if name == "batch":
        ns, ks, _ = W.batch_shapes(npairs)
    else:
        ns, ks = W.serve_shapes(npairs)
    for i, (n, m, e, k) in cache.items():
        assert n == ns[i]
        assert e <= ks[i]
        assert abs(n - m) <= k <= e
    # both files are complete
    assert len(cache) == npairs


@pytest.mark.parametrize("name", ["batch", "serve"])
def test_smallest_pairs_recomputed(orc, name):
    cache = FC.load(name)
    npairs = FC.FILES[name][1]
    if name == "batch":
        ns, ks, sig = W.batch_shapes(npairs)
        seed = 4
    else:
        ns, ks = W.serve_shapes(npairs)
        sig = np.full(npairs, 4)
        seed = 5
    small = sorted(cache, key=lambda i: ns[i] * (ks[i] + 1))[:12]
    for i in small:
        p = W.make_pair(seed, int(ns[i]), int(ks[i]), sigma=int(sig[i]), extra=i + 1)
        assert (p.A.size, p.B.size, p.edits) == cache[i][:3]
        k = orc.lv(p.A, p.B)
        assert k == cache[i][3]
        if p.A.size * p.B.size <= 4_000_000:
            assert orc.dp(p.A, p.B) == k

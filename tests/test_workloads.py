"""The seeded generators: deterministic, and shaped as their recipe says."""
import numpy as np

from paper_2306_17461_gb300 import workloads as W


def test_deterministic():
    a = W.single_small(n=20000, k=30)
    b = W.single_small(n=20000, k=30)
    assert np.array_equal(a.A, b.A) and np.array_equal(a.B, b.B)
    c = W.single_mid(10, n=20000)
    assert not np.array_equal(a.A, c.A)


def test_planted_count_and_lengths():
    p = W.make_pair(50, 100000, 1000, sigma=4)
    assert p.edits == 1000
    assert abs(p.B.size - p.A.size) <= 1000
    assert p.A.max() < 4 and p.B.max() < 4


def test_zipf_shares():
    sym = W.Symbols(zipf_s=1.1)
    x = sym.draw(np.random.default_rng(0), 2_000_000)
    share = np.bincount(x, minlength=256) / x.size
    w = np.arange(1, 257, dtype=np.float64) ** -1.1
    w /= w.sum()
    assert abs(share[0] - 0.2065) < 0.003 and abs(w[0] - 0.2065) < 0.001
    assert np.all(share > 0)
    assert abs((share ** 2).sum() - 0.0635) < 0.002


def test_bursts_cluster():
    rng = W.rng_for(3)
    pos = W.burst_positions(rng, 10**7, 2000)
    assert 1800 <= pos.size <= 2000
    gaps = np.diff(pos)
    # most consecutive edits are a few characters apart (inside a burst)
    assert np.median(gaps) <= 8


def test_batch_shapes():
    ns, ks, sig = W.batch_shapes()
    assert ns.size == 4096 and ns.min() >= 1000 and ns.max() <= 10**6
    assert set(np.unique(sig).tolist()) == {4, 64}
    r = ks / ns
    assert r.min() >= 0 and r.max() <= 0.051


def test_poisson_arrivals():
    t = W.poisson_arrivals(10.0, 5000)
    assert np.all(np.diff(t) > 0)
    assert abs(t[-1] / 5000 - 0.1) < 0.01


def test_lcp_length_pairs_are_skewed_binary_and_seeded():
    from paper_2306_17461_gb300 import workloads as W

    for p0 in (0.5, 0.9, 0.99):
        p = W.lcp_length_pair(200, p0, n=200_000)
        assert set(np.unique(p.A).tolist()) <= {0, 1} and set(np.unique(p.B).tolist()) <= {0, 1}
        assert abs((p.A == 0).mean() - p0) < 0.01
        assert p.edits == 200 and abs(p.B.size - p.A.size) <= 200
        q = W.lcp_length_pair(200, p0, n=200_000)
        assert np.array_equal(p.A, q.A) and np.array_equal(p.B, q.B)


def test_binary_substitution_flips_the_symbol():
    from paper_2306_17461_gb300 import workloads as W

    sym = W.Symbols(p0=0.999)
    old = np.array([0, 1, 0, 0, 1], dtype=np.uint8)
    assert sym.draw_unlike(np.random.default_rng(0), old).tolist() == [1, 0, 1, 1, 0]

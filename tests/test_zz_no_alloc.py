"""The allocation-free prefix hash (ed_prefix_hash_noalloc), for callers
whose memory manager owns every device allocation or who cannot pay for
cudaMalloc / cudaFree on their path.

Checked through the C ABI against the context-based ed_prefix_hash_dev on
the same inputs (integer results: equal bit for bit) and directly against
the oracle's table (the definition of Sec. 3.2 in plain C), on two calls in
a row that share the library's fixed scratch array, at the largest length
the scratch holds (its last look-back descriptor at the array's end), on a
side stream, and for the size limit.  This file is collected last on
purpose, so that a run stopping at the first failure has already run every
other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def test_noalloc_matches_context_entry_point_twice(orc):
    import torch

    from paper_2306_17461_gb300 import binding as ed

    ctx = ed.Context(device=0)
    base = ed.ed_hash_base(ctx.h)
    rng = np.random.default_rng(2024)
    # two calls in a row with different lengths: the second must not see the
    # first call's leftovers in the shared scratch
    for length in (1_000_003, 70_001):
        x = rng.integers(0, 256, length, dtype=np.uint8)
        X = _dev(x)
        want = ed.ed_prefix_hash_dev(ctx.h, X).cpu().numpy().view(np.uint64)
        T = torch.empty(length + 1, dtype=torch.int64, device=X.device)
        ed.ed_prefix_hash_noalloc(X, base, T)
        got = T.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want), length
        assert np.array_equal(got, orc.prefix_hash(x, base)), length
    ctx.close()


def test_noalloc_at_the_length_limit_on_a_side_stream(orc):
    """len == ED_NOALLOC_MAX_LEN: the scan's last descriptor ends exactly at
    the end of the 1 MiB scratch.  Run on a torch side stream, compared with
    the oracle entry by entry."""
    import torch

    from paper_2306_17461_gb300 import binding as ed

    n = ed.ED_NOALLOC_MAX_LEN
    x = np.random.default_rng(7).integers(0, 256, n, dtype=np.uint8)
    base = 1_000_003
    X = _dev(x)
    T = torch.empty(n + 1, dtype=torch.int64, device=X.device)
    side = torch.cuda.Stream()
    ed.ed_prefix_hash_noalloc(X, base, T, stream=side)
    got = T.cpu().numpy().view(np.uint64)
    want = orc.prefix_hash(x, base)
    assert np.array_equal(got, want)
    # the next call, shorter, on the default stream, after the full one
    T2 = torch.empty(1001, dtype=torch.int64, device=X.device)
    ed.ed_prefix_hash_noalloc(X[:1000], base, T2)
    assert np.array_equal(T2.cpu().numpy().view(np.uint64), want[:1001])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_2306_17461_gb300 import binding as ed

    lib = ed.load()
    X = torch.zeros(16, dtype=torch.uint8, device="cuda")
    T = torch.zeros(17, dtype=torch.int64, device="cuda")
    # rejected before any device access: the length alone exceeds the limit
    r = lib.ed_prefix_hash_noalloc(ctypes.c_void_p(X.data_ptr()), ed.ED_NOALLOC_MAX_LEN + 1, 257,
                                   ctypes.c_void_p(T.data_ptr()), None)
    assert r == ed.ED_EINVAL
    # an empty string is accepted and gives T[0] = 0
    assert lib.ed_prefix_hash_noalloc(None, 0, 257, ctypes.c_void_p(T.data_ptr()), None) == ed.ED_OK
    assert int(T[0].item()) == 0
    # the binding refuses a non-contiguous output before the call
    T3 = torch.zeros(34, dtype=torch.int64, device="cuda")[::2]
    with pytest.raises(ValueError):
        ed.ed_prefix_hash_noalloc(X, 257, T3)

"""The allocation-free prefix hash (ed_prefix_hash_noalloc), for callers
whose memory manager owns every device allocation or who cannot pay for
cudaMalloc / cudaFree on their path.

Checked through the C ABI against the context-based ed_prefix_hash_dev on
the same inputs (integer results: equal bit for bit), on two calls in a row
that share the library's fixed scratch array, and for the size limit.  This
file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def test_noalloc_matches_context_entry_point_twice():
    import torch

    from paper_2306_17461_gb300 import binding as ed

    ctx = ed.Context(device=0)
    base = ed.ed_hash_base(ctx.h)
    rng = np.random.default_rng(2024)
    # two calls in a row with different lengths: the second must not see the
    # first call's leftovers in the shared scratch
    for length in (1_000_003, 70_001):
        X = _dev(rng.integers(0, 256, length, dtype=np.uint8))
        want = ed.ed_prefix_hash_dev(ctx.h, X).cpu().numpy().view(np.uint64)
        T = torch.empty(length + 1, dtype=torch.int64, device=X.device)
        ed.ed_prefix_hash_noalloc(X, base, T)
        got = T.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want), length
    ctx.close()


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

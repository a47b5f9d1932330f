"""CPU oracle for exact Levenshtein distance and the Landau-Vishkin frontier.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg may import this package.  The product
path (the CUDA library and its binding) never imports it, and it imports
nothing from the product.

What it computes, with the passage each function follows:

* ``dp``            -- the DP recurrence of Sec. 1 (two rows), the plain
                       definition of the distance.
* ``dp_table``      -- the full DP table, for frontier-definition checks.
* ``lv``            -- Algorithm 1 (Sec. 3.1, Appendix A), diagonal
                       i = x - y, char-by-char LCP; ``nthreads > 1`` runs the
                       diagonals of a round in parallel (OpenMP).
* ``lv_frontiers``  -- the frontiers f_0..f_t of Algorithm 1.
* ``lcp``           -- LCP(A, B, x, y) of Sec. 2, one character at a time.
* ``prefix_hash``   -- T[x] = h(X[1..x]) of Sec. 2 / Sec. 3.2, mod 2^61-1.
* ``hash_lcp``      -- the doubling-then-binary search LCP of Sec. 3.2.
* ``prefix_hash_blocked``, ``get_hash_blocked``, ``hash_lcp_blocked`` --
  the blocked table of Sec. 3.3 (Alg. 2: block prefixes only, GetHash
  extends them by the characters after the last whole block).
* ``many``          -- DP or Algorithm 1 over many pairs (host threads).

The arithmetic lives in ``oracle.c`` (plain C, int64, exact 128-bit
products for the hash); this module only marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
NEG = -(2**63) // 4  # "minus infinity" in frontier dumps
Q = (1 << 61) - 1

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    i64, u64, vp, ci = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
    lib.orc_dp.restype = i64
    lib.orc_dp.argtypes = [vp, i64, vp, i64]
    lib.orc_dp_table.restype = ci
    lib.orc_dp_table.argtypes = [vp, i64, vp, i64, vp]
    lib.orc_lcp.restype = i64
    lib.orc_lcp.argtypes = [vp, i64, vp, i64, i64, i64]
    lib.orc_lv.restype = i64
    lib.orc_lv.argtypes = [vp, i64, vp, i64, i64, ci, vp]
    lib.orc_lv_frontiers.restype = i64
    lib.orc_lv_frontiers.argtypes = [vp, i64, vp, i64, i64, vp]
    lib.orc_many.restype = ci
    lib.orc_many.argtypes = [ci, i64, vp, vp, vp, vp, ci, vp]
    lib.orc_prefix_hash.restype = ci
    lib.orc_prefix_hash.argtypes = [vp, i64, u64, vp]
    lib.orc_range_hash.restype = u64
    lib.orc_range_hash.argtypes = [vp, i64, i64, u64]
    lib.orc_powmod.restype = u64
    lib.orc_powmod.argtypes = [u64, i64]
    lib.orc_hash_lcp.restype = i64
    lib.orc_hash_lcp.argtypes = [vp, i64, vp, i64, u64, i64, i64]
    lib.orc_prefix_hash_blocked.restype = ci
    lib.orc_prefix_hash_blocked.argtypes = [vp, i64, i64, u64, vp]
    lib.orc_get_hash_blocked.restype = u64
    lib.orc_get_hash_blocked.argtypes = [vp, vp, i64, u64, i64]
    lib.orc_hash_lcp_blocked.restype = i64
    lib.orc_hash_lcp_blocked.argtypes = [vp, i64, vp, vp, i64, vp, i64, u64, i64, i64]
    lib.orc_num_threads.restype = ci
    lib.orc_num_threads.argtypes = []
    _lib = lib
    return lib


def _u8(s) -> np.ndarray:
    if isinstance(s, (bytes, bytearray)):
        return np.frombuffer(bytes(s), dtype=np.uint8)
    if isinstance(s, str):
        return np.frombuffer(s.encode("latin-1"), dtype=np.uint8)
    a = np.ascontiguousarray(s, dtype=np.uint8)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


def num_threads() -> int:
    return int(_load().orc_num_threads())


def dp(A, B) -> int:
    """Edit distance by the Sec. 1 recurrence (Theta(nm) time, O(m) space)."""
    a, b = _u8(A), _u8(B)
    r = _load().orc_dp(_ptr(a), a.size, _ptr(b), b.size)
    if r < 0:
        raise MemoryError("oracle dp: allocation failed")
    return int(r)


def dp_table(A, B) -> np.ndarray:
    """Full (n+1) x (m+1) DP table G[x][y] (tiny inputs only)."""
    a, b = _u8(A), _u8(B)
    G = np.empty((a.size + 1, b.size + 1), dtype=np.int64)
    _load().orc_dp_table(_ptr(a), a.size, _ptr(b), b.size, G.ctypes.data_as(ctypes.c_void_p))
    return G


def lcp(A, B, x: int, y: int) -> int:
    a, b = _u8(A), _u8(B)
    return int(_load().orc_lcp(_ptr(a), a.size, _ptr(b), b.size, x, y))


def lv(A, B, max_rounds: int = -1, nthreads: int = 1, with_stats: bool = False):
    """Edit distance by Algorithm 1.  Returns k (or -1 when ``max_rounds``
    stopped it first); with ``with_stats`` also (rounds, extensions)."""
    a, b = _u8(A), _u8(B)
    st = np.zeros(2, dtype=np.int64)
    r = _load().orc_lv(_ptr(a), a.size, _ptr(b), b.size, max_rounds, nthreads,
                       st.ctypes.data_as(ctypes.c_void_p))
    if r == -2:
        raise MemoryError("oracle lv: allocation failed")
    if with_stats:
        return int(r), int(st[0]), int(st[1])
    return int(r)


def lv_frontiers(A, B, t_max: int):
    """(k or -1, F) with F[t, i + t_max] = f_t[i] (NEG where undefined)."""
    a, b = _u8(A), _u8(B)
    F = np.empty((t_max + 1, 2 * t_max + 1), dtype=np.int64)
    k = _load().orc_lv_frontiers(_ptr(a), a.size, _ptr(b), b.size, t_max,
                                 F.ctypes.data_as(ctypes.c_void_p))
    return int(k), F


def many(method: str, pairs, nthreads: int = 0) -> np.ndarray:
    """DP ('dp') or Algorithm 1 ('lv') over a list of (A, B) pairs."""
    code = {"dp": 0, "lv": 1}[method]
    As = [_u8(p[0]) for p in pairs]
    Bs = [_u8(p[1]) for p in pairs]
    aoff = np.zeros(len(pairs) + 1, dtype=np.int64)
    boff = np.zeros(len(pairs) + 1, dtype=np.int64)
    aoff[1:] = np.cumsum([x.size for x in As])
    boff[1:] = np.cumsum([x.size for x in Bs])
    acat = np.concatenate(As) if As else np.zeros(0, np.uint8)
    bcat = np.concatenate(Bs) if Bs else np.zeros(0, np.uint8)
    if acat.size == 0:
        acat = np.zeros(1, np.uint8)
    if bcat.size == 0:
        bcat = np.zeros(1, np.uint8)
    out = np.empty(len(pairs), dtype=np.int64)
    nt = nthreads if nthreads > 0 else (os.cpu_count() or 1)
    _load().orc_many(code, len(pairs), _ptr(acat), _ptr(aoff), _ptr(bcat), _ptr(boff),
                     nt, out.ctypes.data_as(ctypes.c_void_p))
    return out


def prefix_hash(X, base: int) -> np.ndarray:
    """T[0..len] with T[x] = sum_{j<x} (X[j]+1) * base^(x-1-j) mod 2^61-1."""
    x = _u8(X)
    T = np.empty(x.size + 1, dtype=np.uint64)
    _load().orc_prefix_hash(_ptr(x), x.size, base, T.ctypes.data_as(ctypes.c_void_p))
    return T


def range_hash(T: np.ndarray, l: int, length: int, base: int) -> int:
    lib = _load()
    pw = lib.orc_powmod(base, length)
    return int(lib.orc_range_hash(T.ctypes.data_as(ctypes.c_void_p), l, length, pw))


def powmod(base: int, e: int) -> int:
    return int(_load().orc_powmod(base, e))


def hash_lcp(TA: np.ndarray, n: int, TB: np.ndarray, m: int, base: int, x: int, y: int) -> int:
    return int(_load().orc_hash_lcp(TA.ctypes.data_as(ctypes.c_void_p), n,
                                    TB.ctypes.data_as(ctypes.c_void_p), m, base, x, y))


def prefix_hash_blocked(X, b: int, base: int) -> np.ndarray:
    """TB[j] = h(X[0..j*b)) for j = 0..len(X)//b (Sec. 3.3, Alg. 2 Build)."""
    x = _u8(X)
    TB = np.zeros(x.size // b + 1, dtype=np.uint64)
    _load().orc_prefix_hash_blocked(_ptr(x), x.size, b, base, TB.ctypes.data_as(ctypes.c_void_p))
    return TB


def get_hash_blocked(X, TB: np.ndarray, b: int, base: int, i: int) -> int:
    """h(X[0..i)) from the blocked table (Alg. 2 GetHash)."""
    x = _u8(X)
    return int(_load().orc_get_hash_blocked(_ptr(x), TB.ctypes.data_as(ctypes.c_void_p), b, base, i))


def hash_lcp_blocked(A, TA: np.ndarray, B, TB: np.ndarray, b: int, base: int, x: int, y: int) -> int:
    """The LCP search of Sec. 3.2 on blocked tables (Alg. 2 LongestPrefix)."""
    a, bb = _u8(A), _u8(B)
    return int(_load().orc_hash_lcp_blocked(_ptr(a), a.size, TA.ctypes.data_as(ctypes.c_void_p), _ptr(bb), bb.size,
                                            TB.ctypes.data_as(ctypes.c_void_p), b, base, x, y))

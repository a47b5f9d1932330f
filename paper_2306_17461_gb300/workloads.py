"""Seeded synthetic string pairs shaped like the paper's workloads.

This module only draws random inputs.  It holds none of the edit-distance
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

Recipe (Sec. 6, "Tested Algorithms and Datasets"): draw A at random, then
apply k edits, each equally likely an insertion, a deletion or a
substitution.  Positions are distinct and are applied left to right
against the original A, so every edit touches an original character:

* substitution -- A[p] is replaced by a symbol drawn from the same
  distribution, redrawn until it differs;
* deletion     -- A[p] is dropped;
* insertion    -- a drawn symbol is inserted before A[p].

Symbols are the bytes 0..sigma-1.  Zipf(s) symbols use p_i ~ i^-s over
i = 1..256 (byte i-1), drawn through a 65536-entry lookup table (each
symbol's share is rounded to 1/65536).

The five workloads (seed = 20230617 + workload index):

1. ``single_small``  -- n = 10^6, sigma = 4 uniform, 100 uniform edits.
2. ``single_mid``    -- n = 10^8, sigma = 4 uniform, k in {10, 10^3, 10^5}.
3. ``single_large``  -- n = 10^9, Zipf(1.1) over 256 symbols, 10^4 edits
   in bursts: burst lengths Geometric(mean 20), burst starts uniform,
   edits inside a burst at start + cumulative Geometric(mean 4) gaps.
4. ``batch``         -- 4096 pairs, n log-uniform on [10^3, 10^6],
   sigma 4 (even index) or 64 (odd), edit rate log-uniform on
   [10^-4, 5*10^-2], uniform positions.
5. ``serve``         -- 512 pairs, n log-uniform on [10^2, 10^7], sigma 4,
   edit rate log-uniform on [10^-3, 10^-1]; Poisson arrival times.
6. ``lcp_length``    -- the setting of Fig. 4: n = 10^7, k in {10^4,
   5*10^4}, two symbols with P(symbol 0) = p0 skewed so that chance matches
   run long (two random positions agree with probability
   q = p0^2 + (1-p0)^2, a mean run of q / (1 - q)); uniform edits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED0 = 20230617
CHUNK = 1 << 24


@dataclass
class Pair:
    A: np.ndarray
    B: np.ndarray
    edits: int  # number of planted edits (an upper bound on the distance)
    desc: str


def rng_for(index: int, extra: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([SEED0 + index, extra]))


# ---------------------------------------------------------------- symbols
def _zipf_lut(s: float = 1.1, sigma: int = 256) -> np.ndarray:
    w = np.arange(1, sigma + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w / w.sum())
    u = (np.arange(65536, dtype=np.float64) + 0.5) / 65536.0
    return np.minimum(np.searchsorted(cdf, u, side="right"), sigma - 1).astype(np.uint8)


class Symbols:
    """A symbol distribution: uniform over sigma bytes, Zipf over 256, or
    two symbols with P(0) = p0 (through a 65536-entry lookup table)."""

    def __init__(self, sigma: int = 4, zipf_s: float | None = None, p0: float | None = None):
        if p0 is not None:
            self.sigma = 2
            self.lut = (np.arange(65536) >= int(round(p0 * 65536))).astype(np.uint8)
            return
        self.sigma = 256 if zipf_s is not None else sigma
        self.lut = _zipf_lut(zipf_s) if zipf_s is not None else None

    def draw(self, rng: np.random.Generator, size: int) -> np.ndarray:
        out = np.empty(size, dtype=np.uint8)
        for lo in range(0, size, CHUNK):
            hi = min(size, lo + CHUNK)
            if self.lut is None:
                out[lo:hi] = rng.integers(0, self.sigma, hi - lo, dtype=np.uint8)
            else:
                u = rng.integers(0, 65536, hi - lo, dtype=np.uint16)
                out[lo:hi] = self.lut[u]
        return out

    def draw_unlike(self, rng: np.random.Generator, old: np.ndarray) -> np.ndarray:
        """One drawn symbol per entry of ``old``, each different from it."""
        if self.sigma == 2: # the only other symbol
            return (1 - old).astype(np.uint8)
        new = self.draw(rng, old.size)
        bad = new == old
        while bad.any():
            new[bad] = self.draw(rng, int(bad.sum()))
            bad = new == old
        return new


# ---------------------------------------------------------------- edits
def plant(rng: np.random.Generator, A: np.ndarray, positions: np.ndarray,
          sym: Symbols) -> np.ndarray:
    """Apply one random edit (ins/del/sub, equally likely) at each distinct
    sorted position of ``positions`` (indices into A); returns B."""
    pos = np.unique(np.asarray(positions, dtype=np.int64))
    k = pos.size
    if k == 0:
        return A.copy()
    ops = rng.integers(0, 3, k)  # 0 substitute, 1 delete, 2 insert
    subs = sym.draw_unlike(rng, A[pos])
    ins = sym.draw(rng, k)
    pieces = []
    prev = 0
    for p, op, s, c in zip(pos.tolist(), ops.tolist(), subs.tolist(), ins.tolist()):
        pieces.append(A[prev:p])
        if op == 0:
            pieces.append(np.array([s], dtype=np.uint8))
            prev = p + 1
        elif op == 1:
            prev = p + 1
        else:
            pieces.append(np.array([c], dtype=np.uint8))
            prev = p
    pieces.append(A[prev:])
    return np.concatenate(pieces)


def uniform_positions(rng: np.random.Generator, n: int, k: int) -> np.ndarray:
    k = min(k, n)
    if k == 0:
        return np.zeros(0, dtype=np.int64)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)


def burst_positions(rng: np.random.Generator, n: int, k: int,
                    burst_mean: float = 20.0, gap_mean: float = 4.0) -> np.ndarray:
    """Edits in bursts: Geometric(mean burst_mean) edits per burst, burst
    starts uniform on [0, n), edits at start + cumulative Geometric(mean
    gap_mean) gaps.  Duplicates are merged, so the count can fall a little
    short of k."""
    out = []
    total = 0
    while total < k:
        blen = min(int(rng.geometric(1.0 / burst_mean)), k - total)
        start = int(rng.integers(0, n))
        gaps = rng.geometric(1.0 / gap_mean, size=blen)
        out.append(start + np.cumsum(gaps) - gaps[0])
        total += blen
    pos = np.unique(np.concatenate(out)) if out else np.zeros(0, np.int64)
    return pos[pos < n].astype(np.int64)


# ---------------------------------------------------------------- pairs
def make_pair(index: int, n: int, k: int, sigma: int = 4, zipf_s: float | None = None,
              bursts: bool = False, extra: int = 0) -> Pair:
    rng = rng_for(index, extra)
    sym = Symbols(sigma, zipf_s)
    A = sym.draw(rng, n)
    pos = burst_positions(rng, n, k) if bursts else uniform_positions(rng, n, k)
    B = plant(rng, A, pos, sym)
    d = "zipf%.1f" % zipf_s if zipf_s is not None else "sigma%d" % sigma
    return Pair(A, B, int(np.unique(pos).size),
                f"n={n} k_planted={int(np.unique(pos).size)} {d}{' bursts' if bursts else ''}")


def single_small(n: int = 10**6, k: int = 100) -> Pair:
    return make_pair(1, n, k, sigma=4)


def single_mid(k: int, n: int = 10**8) -> Pair:
    return make_pair(2, n, k, sigma=4, extra=k)


def single_large(n: int = 10**9, k: int = 10**4) -> Pair:
    return make_pair(3, n, k, zipf_s=1.1, bursts=True)


def _log_uniform(rng: np.random.Generator, lo: float, hi: float, size: int) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def batch_shapes(npairs: int = 4096, n_lo: float = 1e3, n_hi: float = 1e6,
                 r_lo: float = 1e-4, r_hi: float = 5e-2):
    rng = rng_for(4)
    ns = np.maximum(1, np.round(_log_uniform(rng, n_lo, n_hi, npairs))).astype(np.int64)
    rates = _log_uniform(rng, r_lo, r_hi, npairs)
    ks = np.maximum(0, np.round(ns * rates)).astype(np.int64)
    sig = np.where(np.arange(npairs) % 2 == 0, 4, 64)
    return ns, ks, sig


def batch_pairs(npairs: int = 4096, n_lo: float = 1e3, n_hi: float = 1e6,
                r_lo: float = 1e-4, r_hi: float = 5e-2) -> list[Pair]:
    ns, ks, sig = batch_shapes(npairs, n_lo, n_hi, r_lo, r_hi)
    return [make_pair(4, int(ns[p]), int(ks[p]), sigma=int(sig[p]), extra=p + 1)
            for p in range(npairs)]


def serve_shapes(npairs: int = 512, n_lo: float = 1e2, n_hi: float = 1e7,
                 r_lo: float = 1e-3, r_hi: float = 1e-1):
    rng = rng_for(5)
    ns = np.maximum(1, np.round(_log_uniform(rng, n_lo, n_hi, npairs))).astype(np.int64)
    rates = _log_uniform(rng, r_lo, r_hi, npairs)
    ks = np.maximum(0, np.round(ns * rates)).astype(np.int64)
    return ns, ks


def serve_pairs(npairs: int = 512, n_lo: float = 1e2, n_hi: float = 1e7,
                r_lo: float = 1e-3, r_hi: float = 1e-1) -> list[Pair]:
    ns, ks = serve_shapes(npairs, n_lo, n_hi, r_lo, r_hi)
    return [make_pair(5, int(ns[p]), int(ks[p]), sigma=4, extra=p + 1)
            for p in range(npairs)]


def poisson_arrivals(rate_per_s: float, count: int, seed_extra: int = 0) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process of the given rate."""
    rng = rng_for(5, 10**6 + seed_extra)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, count))


def random_pair(rng: np.random.Generator, n: int, k: int, sigma: int) -> tuple[np.ndarray, np.ndarray]:
    """A small pair for property and parity tests."""
    sym = Symbols(sigma)
    A = sym.draw(rng, n)
    B = plant(rng, A, uniform_positions(rng, n, k), sym)
    return A, B


def lcp_length_pair(k: int, p0: float, n: int = 10**7, extra: int = 0) -> Pair:
    """Fig. 4's setting: n characters over two symbols with P(0) = p0, k
    uniform planted edits (seed 20230617 + 6)."""
    rng = rng_for(6, extra + int(round(p0 * 1e6)) * 7 + k)
    sym = Symbols(p0=p0)
    A = sym.draw(rng, n)
    pos = uniform_positions(rng, n, k)
    B = plant(rng, A, pos, sym)
    return Pair(A, B, int(np.unique(pos).size), f"n={n} k_planted={k} binary p0={p0}")

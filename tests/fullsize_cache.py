"""Reads the oracle's cached distances of the full-size batched (4096) and
served (512) pair sets (tests/golden/*_distances.tsv, written by
tests/golden/make_full_size_cache.py from oracle.lv)."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FILES = {"batch": ("batch4096_distances.tsv", 4096), "serve": ("serve512_distances.tsv", 512)}


def load(name: str) -> dict:
    """index -> (n, m, planted, k)"""
    fname, _ = FILES[name]
    out = {}
    with open(os.path.join(GOLDEN, fname)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            i, n, m, e, k = (int(x) for x in line.split())
            out[i] = (n, m, e, k)
    return out


def complete(name: str) -> bool:
    return len(load(name)) == FILES[name][1]

"""Writes the oracle's distances for the full-size batched and served pair
sets, so that the GPU tests can check every pair without rerunning the
oracle (the served set alone is about 2 * 10^12 diagonal-extensions).

The inputs come from ``paper_2306_17461_gb300.workloads`` (the seeded
generators, no edit-distance arithmetic); every distance comes from
``oracle.lv`` (Algorithm 1 with a char-by-char LCP, Sec. 3.1).  Nothing here
calls the CUDA library.

    python tests/golden/make_full_size_cache.py [--threads T] [batch|serve ...]

Output (one line per pair, resumable: pairs already in a file are skipped):

* ``batch4096_distances.tsv`` -- ``workloads.batch_pairs(4096)``: seed
  20230617 + 4, pair p drawn with extra = p + 1;
* ``serve512_distances.tsv``  -- ``workloads.serve_pairs(512)``: seed
  20230617 + 5, pair p drawn with extra = p + 1.

Columns: pair index, n, m, planted edits, distance.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2306_17461_gb300 import workloads as W  # noqa: E402

SETS = {
    "batch": ("batch4096_distances.tsv", 4096, 4),
    "serve": ("serve512_distances.tsv", 512, 5),
}
# pairs whose estimated work (planted edits squared) is above this run one
# at a time with the diagonals of a round spread over the threads
BIG = 2e9


def header(name: str, npairs: int, seed_index: int) -> str:
    gen = "batch_pairs" if name == "batch" else "serve_pairs"
    return (f"# Distances of workloads.{gen}({npairs}) (seed {W.SEED0} + {seed_index}, pair p drawn\n"
            f"# with extra = p + 1), each computed by oracle.lv (Algorithm 1, Sec. 3.1,\n"
            f"# char-by-char LCP) and written by tests/golden/make_full_size_cache.py.\n"
            f"# columns: index n m planted k\n")


def load(path: str) -> dict[int, tuple[int, int, int, int]]:
    done = {}
    if os.path.exists(path):
        with open(path) as f:
            for line in f:
                if line.startswith("#") or not line.strip():
                    continue
                i, n, m, e, k = (int(x) for x in line.split())
                done[i] = (n, m, e, k)
    return done


def shapes(name: str, npairs: int):
    if name == "batch":
        ns, ks, sig = W.batch_shapes(npairs)
        return ns, ks, sig
    ns, ks = W.serve_shapes(npairs)
    return ns, ks, np.full(npairs, 4)


def make(name: str, p: int, ns, ks, sig) -> W.Pair:
    return W.make_pair(SETS[name][2], int(ns[p]), int(ks[p]), sigma=int(sig[p]), extra=p + 1)


def run(name: str, threads: int) -> None:
    fname, npairs, seed_index = SETS[name]
    path = os.path.join(HERE, fname)
    done = load(path)
    if not os.path.exists(path):
        with open(path, "w") as f:
            f.write(header(name, npairs, seed_index))
    ns, ks, sig = shapes(name, npairs)
    todo = [p for p in range(npairs) if p not in done]
    small = [p for p in todo if float(ks[p]) ** 2 <= BIG]
    big = sorted((p for p in todo if float(ks[p]) ** 2 > BIG), key=lambda p: ks[p])
    t0 = time.time()
    with open(path, "a") as f:
        for lo in range(0, len(small), 256):
            part = small[lo:lo + 256]
            pairs = [make(name, p, ns, ks, sig) for p in part]
            got = oracle.many("lv", [(q.A, q.B) for q in pairs], nthreads=threads)
            for p, q, k in zip(part, pairs, got):
                f.write(f"{p}\t{q.A.size}\t{q.B.size}\t{q.edits}\t{int(k)}\n")
            f.flush()
            print(f"{name}: {lo + len(part)}/{len(small)} small pairs, {time.time() - t0:.0f} s", flush=True)
        for p in big:
            q = make(name, p, ns, ks, sig)
            t1 = time.time()
            k = oracle.lv(q.A, q.B, nthreads=threads)
            f.write(f"{p}\t{q.A.size}\t{q.B.size}\t{q.edits}\t{int(k)}\n")
            f.flush()
            print(f"{name}: pair {p} n={q.A.size} k={k} in {time.time() - t1:.0f} s", flush=True)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("sets", nargs="*", default=["batch", "serve"])
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    oracle.build()
    for s in a.sets:
        run(s, a.threads)


if __name__ == "__main__":
    main()

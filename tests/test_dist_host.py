"""bench.py's multi-process host path on CPU (gloo, world size 2): the
barrier, the max of the elapsed times over ranks and the sum of the units
processed, as rank 0 reports them.  One process per rank, as torchrun would
start them."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank: int, world: int, port: int, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    D = bench.Dist()
    try:
        D.barrier()
        # rank r "took" 1 + r seconds and processed 10 * (r + 1) units
        q.put((rank, D.max(1.0 + rank), D.sum(10.0 * (rank + 1)), D.ws, D.rank))
    finally:
        D.close()


@pytest.mark.timeout(120)
def test_two_rank_reduction_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, mx, sm, ws, rk in out:
        assert ws == 2 and rk == rank
        assert mx == 2.0       # the slowest rank's time
        assert sm == 30.0      # all ranks' units


def test_single_process_defaults():
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    D = bench.Dist()
    assert D.ws == 1 and D.rank == 0 and D.pg is None
    assert D.max(3.5) == 3.5 and D.sum(2.0) == 2.0


def test_lpt_shard_balances_and_covers():
    """Batched pairs go to ranks costliest first, each to the least loaded
    rank: every pair lands on exactly one rank, and no rank's load exceeds
    the lightest one's by more than the largest single cost."""
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    costs = [float(c) for c in [9, 1, 1, 1, 8, 2, 7, 3, 3, 3, 1, 5]]
    for ws in (1, 2, 3, 5):
        parts = bench.lpt_shard(costs, ws)
        assert sorted(i for p in parts for i in p) == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)
    # the batch workload's own shapes: two ranks share the 4096 pairs' cost
    from paper_2306_17461_gb300 import workloads as W

    ns, ks, _ = W.batch_shapes(4096)
    c = [float(ns[p]) + float(ks[p]) ** 2 for p in range(4096)]
    a, b = bench.lpt_shard(c, 2)
    la, lb = sum(c[i] for i in a), sum(c[i] for i in b)
    assert abs(la - lb) <= max(c)
    # round-robin by index would split the same cost far less evenly
    ra, rb = sum(c[0::2]), sum(c[1::2])
    assert abs(la - lb) <= abs(ra - rb)


def _lpt_rank_main(rank: int, world: int, port: int, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_2306_17461_gb300 import workloads as W

    D = bench.Dist()
    try:
        ns, ks, _ = W.batch_shapes(256)
        costs = [float(ns[p]) + float(ks[p]) ** 2 for p in range(256)]
        mine = bench.lpt_shard(costs, D.ws)[D.rank]
        # the ranks agree on the total work without a data-path collective
        total = D.sum(sum(costs[i] for i in mine))
        q.put((D.rank, mine, total, sum(costs)))
    finally:
        D.close()


@pytest.mark.timeout(120)
def test_two_rank_lpt_shards_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_lpt_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    (r0, m0, t0, c0), (r1, m1, t1, c1) = out
    assert (r0, r1) == (0, 1)
    assert sorted(m0 + m1) == list(range(256)) and not set(m0) & set(m1)
    assert t0 == t1 == c0 == c1

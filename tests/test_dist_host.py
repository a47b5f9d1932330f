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

"""Multi-replica bookkeeping of bench.py on CPU (gloo, world size 2): updates are
summed over ranks and the timed region is the slowest rank's."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp

from tests.conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    upd, ms = bench.aggregate_over_ranks(1000 * (rank + 1), 10.0 + 5 * rank, "cpu", world)
    q.put((rank, upd, ms))
    dist.destroy_process_group()


def test_replica_aggregation_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, upd, ms in res:
        assert upd == 3000.0 and ms == 15.0


def test_single_rank_is_identity():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate_over_ranks(7, 3.5, "cpu", 1) == (7.0, 3.5)

"""The N-GPU bench path runs independent replicas (no data-path collective): two
gloo ranks on the CPU check the max-over-ranks timing, the barrier, the per-rank
seeds and the whole-job value."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        slowest = bench.max_over_ranks(ms, world)
        q.put((rank, slowest, bench.replica_seed(rank), bench.replicas_value(slowest, world)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [150.0, 150.0]  # both ranks see the slowest time
    assert out[0][2] != out[1][2]  # each replica solves its own gauge field
    assert out[0][3] == pytest.approx(2 * 1e3 / 150.0)  # two solves per slowest step

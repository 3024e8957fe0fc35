"""The multi-rank path of bench.py (replicas, one per GPU) on CPU with two
gloo ranks: the max-over-ranks timing, the whole-job aggregate, and the
reference arm exiting on ranks other than 0 without work."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    m = bench.reduce_max(local_ms)
    value = bench.aggregate_value(1.0, m * 1e-3, world)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, m, value))


def _reference_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup = 1, 3
    if rank == 0:
        out.put((rank, "skipped"))   # rank 0 would run the oracle; not here
        return
    bench.run_reference(A())         # must return at once on rank 1
    out.put((rank, "returned"))


def _run(fn, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=fn, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return sorted(res)


def test_max_over_ranks_and_aggregate():
    res = _run(_worker)
    for rank, m, value in res:
        assert m == 15.0                       # every rank sees the slowest time
        assert value == pytest.approx(2 / 0.015)  # two replicas' units over that time


def test_reference_arm_runs_on_rank_zero_only():
    res = _run(_reference_worker)
    assert res == [(0, "skipped"), (1, "returned")]

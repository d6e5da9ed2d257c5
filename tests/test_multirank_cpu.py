"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Each rank builds its own replica (no data-path collective); the cross-rank
steps are the barrier around the timed region and the maximum of the ranks'
times, and a rank that dies must make the other rank's next collective fail
instead of hanging."""
import datetime
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port, timeout_s):
    import torch.distributed as dist
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            init_method=f"tcp://127.0.0.1:{port}",
                            timeout=datetime.timedelta(seconds=timeout_s))
    return dist


def _aggregate_rank(rank, world, port, out):
    dist = _init(rank, world, port, 30)
    import bench
    w, r, _ = bench.rank_env()
    assert (w, r) == (world, rank)
    local_ms = [120.0, 250.0][rank]           # the ranks' own timed totals
    dist.barrier()
    total = bench.max_over_ranks(local_ms, world)
    value = bench.job_throughput(world, 131072, 10, total)
    out.put((rank, total, value))
    dist.barrier()
    dist.destroy_process_group()


def _dead_rank(rank, world, port, out):
    dist = _init(rank, world, port, 3)
    if rank == 1:
        # this rank fails between steps and leaves without its collective
        out.put((rank, "left"))
        out.close()
        out.join_thread()      # the message is out before the process ends
        os._exit(0)
    try:
        dist.barrier()
        out.put((rank, "no error"))
    except Exception as e:   # the failure reaches the surviving rank as an error
        out.put((rank, "error: " + type(e).__name__))


def _run(fn, world=2):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=fn, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert not p.is_alive(), "a rank hung"
    res = [out.get(timeout=5) for _ in range(world)]
    return sorted(res, key=lambda x: x[0])


def test_two_ranks_take_the_slowest_time_and_sum_the_points():
    res = _run(_aggregate_rank)
    assert [r[1] for r in res] == [250.0, 250.0]
    expect = 2 * 131072 * 10 / 0.25
    assert all(abs(r[2] - expect) < 1e-6 * expect for r in res)


def test_a_dead_rank_fails_the_survivors_collective():
    res = _run(_dead_rank)
    assert res[1] == (1, "left")
    assert res[0][1].startswith("error"), res[0]

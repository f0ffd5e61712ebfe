"""The multi-GPU path of bench.py on CPU: two gloo ranks, each with its own
shard (no data exchanged), the job timed by the slowest rank and credited
with the work of both -- the weak-scaling aggregation the benchmark reports;
and a rank that leaves before the timing barrier, which must end the other
rank's barrier with an error within the process-group timeout, not hang it."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    d = bench.Dist()
    try:
        assert d.world == world and d.rank == rank
        d.barrier()
        # rank r "took" 10*(r+1) ms for 5 steps over its own 1e9 bits per step
        ms_per_step, gbps = bench.aggregate_throughput(d, 10.0 * (rank + 1), 1e9, 5)
        out_q.put((rank, ms_per_step, gbps))
    finally:
        d.close()


def test_two_rank_weak_scaling_aggregation():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=5) for _ in range(world))
    for rank, ms_per_step, gbps in res:
        assert ms_per_step == pytest.approx(20.0 / 5)          # the slowest rank's time
        assert gbps == pytest.approx(2e9 / (20.0 / 5 / 1e3) / 1e9)   # both ranks' work


def test_single_rank_aggregation_is_local():
    import bench
    os.environ.pop("WORLD_SIZE", None)
    d = bench.Dist()
    ms, gbps = bench.aggregate_throughput(d, 8.0, 4e9, 4)
    assert ms == 2.0 and gbps == pytest.approx(4e9 / 2e-3 / 1e9)


def _leaving_rank_main(rank, world, port, out_q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import time
    import bench
    d = bench.Dist(timeout_s=5.0)
    if rank == 1:
        out_q.put((rank, "left"))       # leaves between steps: never reaches the barrier
        return
    t0 = time.monotonic()
    try:
        d.barrier()
        out_q.put((rank, "barrier passed"))
    except Exception as e:              # the expected outcome: an error, not a hang
        out_q.put((rank, f"error after {time.monotonic() - t0:.1f} s: {type(e).__name__}"))


def test_rank_that_leaves_ends_the_other_ranks_barrier_with_an_error():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_leaving_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung"
    res = dict(q.get(timeout=5) for _ in range(world))
    assert res[1] == "left"
    assert res[0].startswith("error after"), res[0]

"""The multi-GPU path of bench.py is independent replicas: each rank runs its
own sampler; the job's step time is the slowest rank's and the value counts
every rank's particles.  Checked with two gloo ranks on the CPU."""
import os

import pytest
import torch.multiprocessing as mp


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local = [12.5, 20.0][rank]
    t = bench.max_over_ranks(local, world, device="cpu")
    v = bench.job_value(1 << 20, 10, world, t)
    q.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    old = os.environ.get("PYTHONPATH", "")
    os.environ["PYTHONPATH"] = root + (os.pathsep + old if old else "")
    try:
        for p in procs:
            p.start()
        out = sorted(q.get(timeout=120) for _ in procs)
        for p in procs:
            p.join(timeout=60)
    finally:
        os.environ["PYTHONPATH"] = old
        for p in procs:
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    for rank, t, v in out:
        assert t == 20.0
        assert v == pytest.approx((1 << 20) * 10 * 2 / 0.020)


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_value(100, 10, 1, 1000.0) == pytest.approx(1000.0)

"""The multi-rank host logic of bench.py on world-size-2 gloo process groups
(CPU): the max-over-ranks timer, the whole-job rate of weak scaling, the
reference arm's rank rule (rank 0 alone runs the oracle; the others return
without work), and the launch environment read from RANK / WORLD_SIZE /
LOCAL_RANK."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist
    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        env = bench.dist_env()
        # per-rank step times: the slower rank sets the job's time
        t = bench.max_over_ranks(1.5 + rank, world)
        rate = bench.whole_job_rate(1e9, 4, world, t)
        # the reference arm on rank 1 returns before any oracle work
        skipped = None
        if rank == 1:
            class A:
                steps, warmup, gpus = 1, 0, world
            skipped = bench.run_reference(A(), None, None, "w") is None
        tdist.barrier()
        q.put((rank, env, t, rate, skipped))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, t, rate, skipped in res:
        assert env == (rank, 2, rank)
        assert t == 2.5                         # the slower rank's time, on both ranks
        assert rate == pytest.approx(1e9 * 4 * 2 / 2.5 / 1e9)
    assert res[1][4] is True


def test_one_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.whole_job_rate(5.0e10, 10, 1, 0.2) == pytest.approx(2500.0)
